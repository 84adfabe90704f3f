"""Failure paths, on the GPU, in the forms that fault nothing: an allocator
that returns NULL, solver iteration caps lowered to zero, and the
tensor-core kernel's bounded pipeline wait shortened to 2 ms and pointed at
a barrier that nothing arrives at, so that it runs out and the kernel
aborts cleanly.  Each surfaces as a status code at the next synchronising
call, and the library stays usable afterwards (a clean call gives the same
results as before, up to FP32 rounding)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu

ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


@pytest.fixture()
def setup(cuda_lib):
    from paper_2601_11626_gb300 import csvd
    w = synth.scoring_c4(r=32, n_states=2, appends=2, per_state=4, m=512, k_lo=16, k_hi=200,
                         device="cuda")
    states = []
    for blocks in w["states"]:
        st = csvd.IncrSVD(w["m"], w["r"])
        for b in blocks:
            st.append(b)
        states.append(st)
    torch.cuda.synchronize()
    yield csvd, w, states
    csvd.debug_limits()  # defaults, whatever happened
    csvd.lib().csvd_set_allocator(None, None, None)


def _same(got, ref):
    """Two clean runs agree up to FP32 rounding (the order of atomic sums
    differs between runs): E~ within the parity tolerance, flags equal."""
    g, r = got[1], ref[1]
    assert np.all(np.abs(g - r) <= 2e-4 * r + 1e-6 * np.abs(r).max()), (g, r)
    assert np.array_equal(got[2], ref[2])


def _score(csvd, w, states, form):
    sig, tail, paper, acc = csvd.score(states, w["cand_state"], w["candidates"], 0.2, form)
    return sig.cpu().numpy(), tail.cpu().numpy(), acc.cpu().numpy()


def _sync_status(states):
    """The next synchronising call on the state whose status word the
    scoring launch used (the first one)."""
    states[0].sigma()


def test_allocator_returning_null_gives_oom(setup):
    csvd, w, states = setup
    ref = _score(csvd, w, states, "mixed")
    calls = []

    @ALLOC
    def no_memory(nbytes, stream, ctx):
        calls.append(nbytes)
        return None

    @FREE
    def no_free(ptr, stream, ctx):
        pass

    lib = csvd.lib()
    assert lib.csvd_set_allocator(ctypes.cast(no_memory, ctypes.c_void_p),
                                  ctypes.cast(no_free, ctypes.c_void_p), None) == 0
    with pytest.raises(csvd.CsvdError) as e:
        _score(csvd, w, states, "mixed")
    assert e.value.status == csvd.Status.ERR_OOM
    assert calls  # the workspace was requested through the callback
    assert lib.csvd_set_allocator(None, None, None) == 0
    got = _score(csvd, w, states, "mixed")
    _same(got, ref)
    _sync_status(states)


@pytest.mark.parametrize("form,caps", [("mixed", (-1, 0)), ("plain", (0, -1)),
                                       ("gram_fp32", (-1, 0))])
def test_zero_iteration_caps_give_not_converged(setup, form, caps):
    csvd, w, states = setup
    ref = _score(csvd, w, states, form)
    _sync_status(states)
    csvd.debug_limits(jacobi_sweeps=caps[0], solver_iters=caps[1])
    _score(csvd, w, states, form)
    with pytest.raises(csvd.CsvdError) as e:
        _sync_status(states)
    assert e.value.status == csvd.Status.ERR_NOT_CONVERGED
    csvd.debug_limits()
    got = _score(csvd, w, states, form)
    _sync_status(states)
    _same(got, ref)


def test_pipeline_waits_that_give_up_give_timeout(setup):
    csvd, w, states = setup
    ref = _score(csvd, w, states, "mixed")
    _sync_status(states)
    csvd.debug_limits(wait_ns=2_000_000, stall_gram=True)   # a barrier nothing arrives at, 2 ms
    _score(csvd, w, states, "mixed")
    with pytest.raises(csvd.CsvdError) as e:
        _sync_status(states)
    assert e.value.status == csvd.Status.ERR_TIMEOUT
    csvd.debug_limits()
    got = _score(csvd, w, states, "mixed")
    _sync_status(states)
    _same(got, ref)
