"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (derived from FP32 arithmetic; the same for the plain and the
mixed form, whose Gram products carry FP32-level accuracy and whose small
tails are re-solved in FP64):
* sigma~: |d sigma_j| <= 1e-5 sigma_j + 2e-6 sigma_1.  The second term is
  the normwise floor of FP32 products (~30 u sigma_1): a singular value far
  below sigma_1 cannot be resolved better than that from FP32 data.  For the
  Gram-eigenvalue forms the floor sits on sigma^2 instead:
  |d sigma_j^2| <= 2e-5 sigma_j^2 + 8 u sigma_1^2 is accepted as well.
* tail: E~ within 1e-4 relative, i.e. |d E~^2| <= 2e-4 E~^2, plus a floor of
  4 u ||M||^2 on E~^2 (u = 2^-24), the rounding of FP32 data of total energy
  ||M||^2; it matters only for tails below ~1.5e-2 ||M||.
* accept flags identical except for merges whose relative estimate lies
  within 1e-3 (relative) of eps; those are listed (printed) and checked to
  lie in that window on the GPU side too.

Every merge evaluation and every append is compared from identical states:
the oracle's state is rounded to FP32 and loaded into the GPU state.  A
free-running GPU trajectory is not compared value by value with the
oracle's: where a truncation cuts through near-equal eigenvalues (a dense
noise floor, repeated latent spectra) the retained basis is ill-conditioned
and FP32 and FP64 trajectories part, both valid; it is checked against
invariants that hold for any valid trajectory instead.
"""
import math

import numpy as np
import pytest
import torch

from oracle import bounds as obounds
from oracle import cluster as ocluster
from oracle import exact as oexact
from oracle import incremental as oinc
from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
TAIL_RTOL = 1e-4
TAIL_FLOOR_U = 4.0
SIGMA_RTOL, SIGMA_FLOOR = 1e-5, 2e-6
GRAM_FLOOR_U = 8.0
BOUNDARY_RTOL = 1e-3


def _np(t):
    return t.detach().cpu().double().numpy()


def _check_sigma(got, want, gram=False):
    """``gram``: sigma~ from eigenvalues of a Gram (the mixed forms), whose
    normwise FP32 floor lies on sigma^2: GRAM_FLOOR_U u sigma_1^2 on
    sigma_j^2, which exceeds 2e-6 sigma_1 on sigma_j below sigma_j ~ 0.06
    sigma_1."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, (got.shape, want.shape)
    if want.size == 0:
        return
    err = np.abs(got - want)
    bound = SIGMA_RTOL * want + SIGMA_FLOOR * want[0]
    if gram:
        ok_sq = np.abs(got ** 2 - want ** 2) <= 2 * SIGMA_RTOL * want ** 2 + \
            GRAM_FLOOR_U * U32 * want[0] ** 2
        bound = np.where(ok_sq, np.inf, bound)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"sigma mismatch at {bad[:8]}: got {got[bad[:8]]} want {want[bad[:8]]}"


def _check_tail(got_sq, want_sq, energy=0.0, rtol=TAIL_RTOL, floor_u=TAIL_FLOOR_U):
    """|E~^2_gpu - E~^2_oracle| <= 2 rtol E~^2 + floor_u u ||M||^2 (``energy``
    is ||M||^2 after the merge)."""
    g, w = max(got_sq, 0.0), max(want_sq, 0.0)
    bound = 2.0 * rtol * w + floor_u * U32 * max(energy, 0.0)
    assert abs(g - w) <= bound, (g, w, abs(g - w), bound, abs(math.sqrt(g) - math.sqrt(w)) /
                                 max(math.sqrt(w), 1e-300))


@pytest.fixture(scope="module")
def csvd(cuda_lib):
    from paper_2601_11626_gb300 import csvd as mod
    return mod


def _round_state(ost):
    """Round the oracle state to FP32 in place (both sides start identical)."""
    ost.Q = ost.Q.astype(np.float32).astype(np.float64)
    ost.s = ost.s.astype(np.float32).astype(np.float64)
    return ost


def _load(csvd, ost):
    g = csvd.IncrSVD(ost.m, ost.r)
    U = torch.tensor(ost.Q, dtype=torch.float32, device="cuda")
    g.load(U, ost.s.astype(np.float32), ost.energy, ost.discarded)
    return g


def _oracle_states(m, r, groups):
    out = []
    for blocks in groups:
        c = oinc.IncrementalSVD(m, r)
        for b in blocks:
            c.append(b)
        out.append(_round_state(c))
    return out


# ------------------------------------------------- one merge evaluation
def _compare_scores(csvd, gst, cst, cand_state, cands, eps, precision):
    """Every candidate against the oracle; returns the boundary merges (those
    whose relative oracle estimate lies within BOUNDARY_RTOL of eps), which are
    printed: their accept flags may differ, and the GPU's estimate must lie
    within the same window widened by the tail tolerance."""
    sig, tail, paper, acc = csvd.score(gst, cand_state, cands, eps, precision)
    sig, tail, paper, acc = _np(sig), _np(tail), _np(paper), acc.cpu().numpy()
    boundary = []
    for i, (si, b) in enumerate(zip(cand_state, cands)):
        s_o, t_o, a_o, nxt = cst[si].evaluate(b.cpu(), eps)
        _check_sigma(sig[i, :len(s_o)], s_o, gram=precision != "plain")
        _check_tail(tail[i], nxt[3], nxt[2])
        rel = math.sqrt(t_o / nxt[2]) if nxt[2] > 0 else 0.0
        if abs(rel - eps) <= BOUNDARY_RTOL * eps:
            boundary.append((i, rel))
            rel_gpu = math.sqrt(max(tail[i], 0.0) / nxt[2])
            assert abs(rel_gpu - eps) <= 2 * BOUNDARY_RTOL * eps, (i, rel, rel_gpu)
        elif bool(acc[i]) != a_o:
            raise AssertionError(f"accept flag differs at {i}: gpu {acc[i]} oracle {a_o}")
    if boundary:
        print(f"boundary merges at eps={eps} ({precision}): {boundary}")
    return boundary


@pytest.mark.parametrize("precision", ["plain", "mixed", "gram_fp32"])
def test_score_c1_eps_005(csvd, precision):
    """The small recipe at its threshold eps = 0.05: states of one latent
    subspace (blocks j, j + 4), candidates of the same subspace (tails of
    ~1.5% of ||M||, accepted) and of another (rejected)."""
    col = synth.small_c1()
    m, r, eps = col.m, col.meta["r"], col.meta["eps"]
    cst = _oracle_states(m, r, [[col.blocks[c], col.blocks[c + 4]] for c in range(4)])
    gst = [_load(csvd, c) for c in cst]
    pairs = [(i, i % 4) for i in range(8, 16)] + [(i, (i + 1) % 4) for i in range(8, 16)]
    cands = [col.blocks[i].cuda() for i, _ in pairs]
    _compare_scores(csvd, gst, cst, [s for _, s in pairs], cands, eps, precision)


@pytest.mark.parametrize("precision", ["plain", "mixed", "gram_fp32"])
def test_score_c2_eps_grid(csvd, precision):
    """The mid-size recipe at eps in {0.02, 0.05, 0.1}: states of one latent
    subspace (1 and 3 blocks), candidates of the same subspace and of others."""
    col = synth.mid_c2(n_blocks=112)
    m, r = col.m, col.meta["r"]
    cst = _oracle_states(m, r, [[col.blocks[0]], [col.blocks[1], col.blocks[17], col.blocks[33]]])
    gst = [_load(csvd, c) for c in cst]
    pairs = [(16 * j, 0) for j in range(1, 7)] + [(16 * j + 1, 1) for j in range(3, 7)]
    pairs += [(i, i % 2) for i in range(100, 106)]
    cands = [col.blocks[i].cuda() for i, _ in pairs]
    for eps in (0.02, 0.05, 0.1):
        _compare_scores(csvd, gst, cst, [s for _, s in pairs], cands, eps, precision)


@pytest.mark.parametrize("precision", ["plain", "mixed", "gram_fp32"])
def test_score_mid_size(csvd, precision):
    col = synth.mid_c2(n_blocks=40)
    m, r = col.m, col.meta["r"]
    cst = _oracle_states(m, r, [col.blocks[0:4], col.blocks[16:19]])
    gst = [_load(csvd, c) for c in cst]
    cands = [b.cuda() for b in col.blocks[20:36]]
    cand_state = [i % 2 for i in range(len(cands))]
    for eps in (0.02, 0.05, 0.1, 0.2):
        _compare_scores(csvd, gst, cst, cand_state, cands, eps, precision)


@pytest.mark.parametrize("precision", ["plain", "mixed"])
def test_score_uneven_large_cores(csvd, precision):
    """Uneven widths in [16, 512] at m = 2048: cores up to 576 x 576 spill
    to global memory before moving on-chip; ragged widths exercise every
    tile tail of the tensor-core Gram."""
    w = synth.scoring_c4(r=64, n_states=3, appends=3, per_state=5, device="cuda")
    m, r = w["m"], w["r"]
    cst = _oracle_states(m, r, w["states"])
    gst = [_load(csvd, c) for c in cst]
    cands = w["candidates"]
    ks = [c.shape[1] for c in cands]
    assert min(ks) < 160 < 330 < max(ks)
    _compare_scores(csvd, gst, cst, w["cand_state"], cands, 0.25, precision)


def test_score_eigen_core_layout_boundaries(csvd):
    """Widths that put the core size n = r_t + k on every edge of the
    mixed-form eigen core's layouts: the launch classes (n <= 192, <= 320,
    larger), the last core held wholly on-chip (448) and the first with a
    global tile column (449), the largest (576), single-tile and one-row
    cores, and ragged tile tails on both sides of each edge."""
    w = synth.scoring_c4(r=64, n_states=1, appends=3, per_state=1, device="cuda")
    m, r = w["m"], w["r"]
    cst = _oracle_states(m, r, w["states"])
    gst = [_load(csvd, c) for c in cst]
    rt = int(gst[0].rank)
    assert rt == 64
    ns = [65, 66, 95, 96, 97, 160, 191, 192, 193, 224, 225, 319, 320, 321, 447, 448, 449, 480,
          481, 575, 576]
    widths = [n - rt for n in ns]
    raw = synth.random_blocks(m, widths, seed=21, decay=0.95, device="cuda")
    # energies comparable to the state's, so that every tail stays a few
    # percent of ||M||^2 (the mixed form's tail floor is ~1e-6 ||M||^2)
    raw = [b * math.sqrt(2000.0 / float((b.double() ** 2).sum())) for b in raw]
    blocks = synth.pack_blocks(raw, ld_align=8)[0]
    # mix in latent-subspace blocks so that some merges are accepted
    blocks = list(blocks) + list(w["candidates"])
    _compare_scores(csvd, gst, cst, [0] * len(blocks), blocks, 0.25, "mixed")


def test_score_one_column_arrowhead(csvd):
    """One-column candidates in the mixed form (the arrowhead core) against the
    oracle: a fresh state (r_t = 0), truncating states with r_t = 24 and
    r_t = 128 (the largest arrowhead), r_t = 160 (past it, the general core),
    and a state that fills every row (no new direction, k' = 0).  Columns are
    random, inside the span of U (plus a little noise), zero, and strided
    views of a wider matrix; two-column candidates ride in the same batch."""
    m = 768
    specs = [(32, []), (24, [16, 24]), (128, [96, 64]), (160, [120, 80])]
    cst, gst = [], []
    for r, widths in specs:
        raw = [b.cpu() for b in synth.random_blocks(m, widths, seed=r, decay=0.97)] if widths else []
        cst += _oracle_states(m, r, [raw])
        gst.append(_load(csvd, cst[-1]))
    assert [int(g.rank) for g in gst] == [0, 24, 128, 160]
    gen = torch.Generator().manual_seed(5)
    cands, cand_state = [], []
    scales = [math.sqrt(max(c.energy, 1.0) / m) for c in cst]
    wide = torch.randn(m, 9, generator=gen, dtype=torch.float64)
    wide = (wide * torch.tensor(scales + [1.0] * (9 - len(scales)))).float().cuda()
    for si, c in enumerate(cst):
        Q = torch.tensor(c.Q, dtype=torch.float64)
        scale = scales[si]
        cols = [torch.randn(m, 1, generator=gen, dtype=torch.float64) * scale]
        if c.Q.shape[1] > 0:
            w = torch.randn(c.Q.shape[1], 1, generator=gen, dtype=torch.float64)
            inspan = Q @ (w * torch.tensor(c.s[:, None]))
            cols.append(inspan + 1e-3 * scale * torch.randn(m, 1, generator=gen, dtype=torch.float64))
            cols.append(torch.zeros(m, 1, dtype=torch.float64))
        for x in cols:
            cands.append(x.float().cuda())
            cand_state.append(si)
        cands.append(wide[:, si:si + 1])
        cand_state.append(si)
        cands.append((torch.randn(m, 2, generator=gen, dtype=torch.float64) * scale).float().cuda())
        cand_state.append(si)
    assert any(b.shape[1] == 1 and b.stride(0) > 1 for b in cands)
    for eps in (0.1, 0.3):
        _compare_scores(csvd, gst, cst, cand_state, cands, eps, "mixed")
    # every row filled: r_t = r = m, so a new column adds no direction
    ms = 96
    full = _oracle_states(ms, ms, [[b.cpu() for b in synth.random_blocks(ms, [60, 50], seed=3)]])
    gfull = [_load(csvd, full[0])]
    assert int(gfull[0].rank) == ms
    col = [(torch.randn(ms, 1, generator=gen, dtype=torch.float64)).float().cuda() for _ in range(3)]
    _compare_scores(csvd, gfull, full, [0, 0, 0], col, 0.2, "mixed")


def test_score_columns_against_oracle(csvd):
    """``csvd_score_columns``: one-column candidates as the rows of one
    matrix (row pitch > m), states with r_t = 0, 24, 128 and 160 (the last
    through the general mixed path), runs of one state of lengths 1 to 7
    between interleaved rows, each row checked against the oracle."""
    m = 768
    specs = [(32, []), (24, [16, 24]), (128, [96, 64]), (160, [120, 80])]
    cst, gst = [], []
    for r, widths in specs:
        raw = [b.cpu() for b in synth.random_blocks(m, widths, seed=r + 1, decay=0.97)] if widths else []
        cst += _oracle_states(m, r, [raw])
        gst.append(_load(csvd, cst[-1]))
    assert [int(g.rank) for g in gst] == [0, 24, 128, 160]
    cand_state = [1] * 7 + [2] * 5 + [0] * 2 + [3] * 4 + [0, 1, 2, 3] * 3 + [2] * 1 + [1] * 6
    n = len(cand_state)
    gen = torch.Generator().manual_seed(9)
    rows = []
    for j, si in enumerate(cand_state):
        c = cst[si]
        scale = math.sqrt(max(c.energy, 1.0) / m)
        x = torch.randn(m, generator=gen, dtype=torch.float64) * scale
        if j % 3 == 0 and c.Q.shape[1] > 0:   # mostly inside the state's span
            w = torch.randn(c.Q.shape[1], generator=gen, dtype=torch.float64)
            x = torch.tensor(c.Q) @ (w * torch.tensor(c.s)) + 1e-2 * x
        rows.append(x)
    Xpad = torch.zeros(n, m + 12, dtype=torch.float32, device="cuda")
    Xpad[:, :m] = torch.stack(rows).float().cuda()
    Xt = Xpad[:, :m]
    assert Xt.stride(0) == m + 12
    for eps in (0.1, 0.3):
        sig, tail, paper, acc = csvd.score_columns(gst, cand_state, Xt, eps)
        sig, tail, acc = _np(sig), _np(tail), acc.cpu().numpy()
        for j, si in enumerate(cand_state):
            s_o, t_o, a_o, nxt = cst[si].evaluate(Xt[j].reshape(m, 1).cpu(), eps)
            _check_sigma(sig[j, :len(s_o)], s_o, gram=True)
            _check_tail(tail[j], nxt[3], nxt[2])
            if abs(math.sqrt(t_o / nxt[2]) - eps) > 1e-3 * eps:
                assert bool(acc[j]) == a_o, (j, acc[j], a_o)


def test_score_simt_and_tensor_gram_agree(csvd):
    """The same candidates through the tensor-core Gram (16-byte aligned rows)
    and the SIMT fallback (odd leading dimension) against the oracle."""
    col = synth.mid_c2(n_blocks=12)
    m, r = col.m, col.meta["r"]
    cst = _oracle_states(m, r, [col.blocks[0:3]])
    gst = [_load(csvd, cst[0])]
    raw = [b[:, :k] for b, k in zip(col.blocks[4:10], (13, 37, 64, 101, 127, 128))]
    aligned, _ = synth.pack_blocks([x.cuda() for x in raw], ld_align=8)
    odd, _ = synth.pack_blocks([x.cuda() for x in raw], ld_align=1)
    odd = [x if x.stride(0) % 4 else torch.nn.functional.pad(x, (0, 1))[:, :x.shape[1]] for x in odd]
    assert any(x.stride(0) % 4 for x in odd)
    for cands in (aligned, odd):
        _compare_scores(csvd, gst, cst, [0] * len(cands), cands, 0.2, "mixed")


def test_score_empty_state_gives_block_spectrum(csvd):
    """A first append scored from an empty state is the rank-r SVD of the
    block (Alg. 3 step 1)."""
    blocks = synth.random_blocks(64, [20, 37], seed=6, decay=0.85)
    for precision in ("plain", "mixed"):
        st = csvd.IncrSVD(64, 10)
        sig, tail, _, _ = csvd.score([st], [0, 0], [b.cuda() for b in blocks], 0.1, precision)
        for i, b in enumerate(blocks):
            s = np.linalg.svd(b.double().numpy(), compute_uv=False)
            _check_sigma(_np(sig)[i, :10], s[:10], gram=precision == "mixed")
            _check_tail(float(tail[i]), float(np.sum(s[10:] ** 2)), float(np.sum(s ** 2)))


def test_score_bf16_blocks_mixed(csvd):
    blocks = synth.random_blocks(128, [40, 64], seed=7, decay=0.9)
    bb = [b.to(torch.bfloat16) for b in blocks]
    st = csvd.IncrSVD(128, 16)
    sig, tail, _, _ = csvd.score([st], [0, 0], [b.cuda() for b in bb], 0.1, "mixed")
    for i, b in enumerate(bb):
        s = np.linalg.svd(b.double().numpy(), compute_uv=False)
        _check_sigma(_np(sig)[i, :16], s[:16], gram=True)
        _check_tail(float(tail[i]), float(np.sum(s[16:] ** 2)), float(np.sum(s ** 2)))


# ----------------------------------------------------- incremental append
def test_append_one_step_from_identical_state(csvd):
    col = synth.mid_c2(n_blocks=8)
    m, r = col.m, col.meta["r"]
    ost = _oracle_states(m, r, [col.blocks[0:5]])[0]
    st = _load(csvd, ost)
    st.append(col.blocks[5].cuda())
    ost.append(col.blocks[5])
    _check_sigma(st.sigma(), ost.s)
    t = st.tail_error()
    _check_tail(t["tail_sq"], ost.tail_sq_discard(), ost.energy)
    assert math.isclose(t["energy"], ost.energy, rel_tol=1e-6)
    U = _np(st.basis())
    assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 2e-5


def _run_pair(csvd, blocks, m, r, precision="plain"):
    """(1) Step parity along the oracle's trajectory: before every append the
    oracle's state (rounded to FP32) is loaded into a GPU state, and the
    step's results are compared.  (2) A free-running GPU trajectory is
    checked at every step against invariants of any valid trajectory:
    sigma~_j <= sigma_j(M) (the retained Gram never exceeds the true one),
    E~ >= E_r(M) (the plug-in estimate is never below the true tail), and
    the energy."""
    free = csvd.IncrSVD(m, r, precision)
    ost = oinc.IncrementalSVD(m, r)
    for t, b in enumerate(blocks):
        _round_state(ost)
        g = _load(csvd, ost) if t > 0 else csvd.IncrSVD(m, r, precision)
        g.append(b.cuda())
        ost.append(b)
        _check_sigma(g.sigma(), ost.s)
        te = g.tail_error()
        _check_tail(te["tail_sq"], ost.tail_sq_discard(), ost.energy)
        g.close()
        free.append(b.cuda())
        s = free.sigma()
        tf = free.tail_error()
        ex = oexact.singular_values(blocks[:t + 1])
        assert np.all(s <= ex[:len(s)] * (1 + 2e-5) + 2e-6 * ex[0])
        assert tf["tail_sq"] >= oexact.tail_sq(blocks[:t + 1], r) * (1 - 2e-4) - 1e-12 * ost.energy
        assert math.isclose(tf["energy"], ost.energy, rel_tol=1e-6)
    U = _np(free.basis())
    assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-4


def test_incremental_small(csvd):
    col = synth.small_c1()
    _run_pair(csvd, col.blocks, col.m, col.meta["r"])


def test_incremental_mid_size(csvd):
    col = synth.mid_c2(n_blocks=12)
    _run_pair(csvd, col.blocks, col.m, col.meta["r"])


def test_incremental_gapped_sequence(csvd):
    """Blocks from 3 latent subspaces with a strong head of 128 directions and
    r = 128; the free-running trajectory ends on the exact top-128 values."""
    w = synth.grad_c5(n_blocks=8, m=512, k=64)
    _run_pair(csvd, w["fd"], 512, 128)


@pytest.mark.parametrize("m,widths,r", [
    (32, [1, 1, 1, 1, 1], 3),          # k = 1 (rank-one appends)
    (16, [2, 2, 2], 12),                # r above the total rank
    (32, [24, 24, 24], 16),             # r_t + k > m: kp = m - r_t
    (40, [7, 33, 5, 64], 9),            # ragged widths, k > m
    (64, [130], 64),                    # single block wider than two GEMM tiles
])
def test_incremental_edge_shapes(csvd, m, widths, r):
    blocks = synth.random_blocks(m, widths, seed=3, decay=0.8)
    _run_pair(csvd, blocks, m, r)


def test_incremental_padded_leading_dimension(csvd):
    blocks = synth.random_blocks(48, [5, 9, 13], seed=4, decay=0.9)
    views, pool = synth.pack_blocks([b.cuda() for b in blocks], ld_align=16)
    st = csvd.IncrSVD(48, 6)
    ost = oinc.IncrementalSVD(48, 6)
    for v, b in zip(views, blocks):
        assert v.stride(0) == 16
        st.append(v)
        ost.append(b)
    _check_sigma(st.sigma(), ost.s)


def test_zero_block(csvd):
    st = csvd.IncrSVD(20, 4)
    ost = oinc.IncrementalSVD(20, 4)
    for b in synth.random_blocks(20, [3], seed=5) + [torch.zeros(20, 4)]:
        st.append(b.cuda())
        ost.append(b)
    _check_sigma(st.sigma(), ost.s)
    _check_tail(st.tail_error()["tail_sq"], ost.tail_sq_discard(), ost.energy)


def test_state_roundtrip(csvd):
    """Export (basis, sigma, tails) and load into a fresh state: appending
    the next block gives the same result as the original state."""
    col = synth.mid_c2(n_blocks=6)
    a = csvd.IncrSVD(col.m, 64)
    for b in col.blocks[:4]:
        a.append(b.cuda())
    t = a.tail_error()
    b2 = csvd.IncrSVD(col.m, 64).load(a.basis(), a.sigma(), t["energy"], t["tail_sq"])
    a.append(col.blocks[4].cuda())
    b2.append(col.blocks[4].cuda())
    np.testing.assert_array_equal(a.sigma(), b2.sigma())
    assert a.tail_error()["tail_sq"] == b2.tail_error()["tail_sq"]


# ----------------------------------------------------------------- bounds
def test_bounds_small(csvd):
    col = synth.small_c1()
    r = col.meta["r"]
    got = csvd.bounds([b.cuda() for b in col.blocks], r)
    w, res, plug, en = obounds.all_bounds(col.blocks, r)
    assert math.isclose(got["energy"], en, rel_tol=1e-6)
    _check_tail(got["weyl_sq"], w, en)
    _check_tail(got["residual_sq"], res, en)
    ex = oexact.tail_sq(col.blocks, r)
    for key in ("weyl_sq", "residual_sq", "plugin_sq"):
        assert got[key] >= ex * (1 - 2e-4)


def test_bounds_gapped_plugin(csvd):
    w = synth.grad_c5(n_blocks=8, m=512, k=64)
    got = csvd.bounds([b.cuda() for b in w["fd"]], 128)
    wb, res, plug, en = obounds.all_bounds(w["fd"], 128)
    _check_tail(got["weyl_sq"], wb, en)
    _check_tail(got["residual_sq"], res, en)
    _check_tail(got["plugin_sq"], plug, en)


# ------------------------------------------------------------- clustering
def _boundary_in_log(log, eps, rtol=1e-3):
    """Logged evaluations whose relative estimate lies within rtol of eps."""
    out = []
    for entry in log:
        _, _, b2, energy, _ = entry
        if energy > 0 and abs(math.sqrt(b2 / energy) - eps) <= rtol * eps:
            out.append((entry[0], entry[1], math.sqrt(b2 / energy)))
    return out


def _labels(clusters, n):
    lab = [0] * n
    for c, mem in enumerate(clusters):
        for j in mem:
            lab[j] = c
    return lab


@pytest.mark.parametrize("algo,mode", [("weyl", "frobenius"), ("residual", "frobenius"),
                                       ("residual", "residual"), ("approx", "frobenius"),
                                       ("approx", "residual")])
@pytest.mark.parametrize("precision", ["plain", "mixed"])
def test_cluster_small(csvd, algo, mode, precision):
    if algo == "residual" and precision == "mixed":
        pytest.skip("Alg. 2 has no mixed form")
    col = synth.small_c1()
    r, eps = col.meta["r"], col.meta["eps"]
    got = csvd.cluster([b.cuda() for b in col.blocks], r, eps, algo, mode, precision)
    want = ocluster.cluster(col.blocks, r, eps, algo, mode)
    # every GPU cluster meets the constraint by the exact SVD (Alg. 1/2 by
    # their theorems, Alg. 3 because its estimate never falls below E_r)
    for c in range(got["n_clusters"]):
        mem = [j for j, l in enumerate(got["labels"]) if l == c]
        assert oexact.rel_error([col.blocks[j] for j in mem], r) <= eps * (1 + 1e-4)
    boundary = _boundary_in_log(want["log"], eps)
    if boundary:
        print(f"boundary merges ({algo}, {mode}, {precision}): {boundary}")
        pytest.skip("a merge lies within 1e-3 of the threshold (listed above)")
    assert got["labels"] == _labels(want["clusters"], len(col.blocks))
    assert math.isclose(got["compression_ratio"], want["compression_ratio"], rel_tol=1e-12)
    for c in range(got["n_clusters"]):
        _check_tail(got["estimate_sq"][c], want["estimate_sq"][c], want["energy"][c])


@pytest.mark.parametrize("algo,mode", [("approx", "frobenius"), ("approx", "residual"),
                                       ("weyl", "frobenius")])
def test_cluster_gapped(csvd, algo, mode):
    """Alg. 3 (and Alg. 1) on blocks from latent subspaces with a strong head
    (merges happen), mixed form."""
    w = synth.grad_c5(n_blocks=12, m=256, k=32)
    blocks = w["blocks"]
    r, eps = 48, 0.2
    got = csvd.cluster([b.cuda() for b in blocks], r, eps, algo, mode, "mixed")
    want = ocluster.cluster(blocks, r, eps, algo, mode)
    if algo == "approx":
        assert len(want["clusters"]) < len(blocks)
    boundary = _boundary_in_log(want["log"], eps)
    if boundary:
        print(f"boundary merges ({algo}, {mode}): {boundary}")
        pytest.skip("boundary merge (listed above)")
    assert got["labels"] == _labels(want["clusters"], len(blocks))


@pytest.mark.parametrize("mode,eps", [("frobenius", 0.2), ("residual", 0.24)])
def test_cluster_one_column_many_blocks(csvd, mode, eps):
    """Alg. 3 on 600 one-column blocks from six latent 5-dim subspaces
    (mixed form, so every merge is scored on the arrowhead core): more
    candidates than one scoring chunk, accepts spread through the scan, and
    clusters of up to 47 (frobenius) and 167 (residual order) members;
    labels equal the oracle's.  The scan makes over 10^4 evaluations, so the
    boundary window is the mixed form's own resolution with margin: a tail
    error of 1e-6 ||M||^2 moves sqrt(E~^2 / ||M||^2) by at most
    0.5e-6 / eps^2 (1.25e-5 at eps = 0.2) relative; evaluations within 5e-5
    of eps skip the test (none at these eps)."""
    m, d, K = 64, 5, 600
    bases = synth.latent_bases(m, d, 6, 11)
    spec = [0.8 ** i for i in range(d)]
    blocks, _, _ = synth.latent_mixture(m, [1] * K, bases, spec, 3e-2, 12, w_max=0.2)
    r = 8
    got = csvd.cluster([b.cuda() for b in blocks], r, eps, "approx", mode, "mixed")
    want = ocluster.cluster(blocks, r, eps, "approx", mode)
    assert max(len(c) for c in want["clusters"]) > 30
    boundary = _boundary_in_log(want["log"], eps, rtol=5e-5)
    if boundary:
        print(f"evaluations within 5e-5 of eps: {boundary}")
        pytest.skip("an evaluation lies within 5e-5 of the threshold (listed above)")
    assert got["labels"] == _labels(want["clusters"], K)


# ------------------------------------------------------------ gradients
def test_tail_grad_matches_oracle(csvd):
    w = synth.grad_c5(n_blocks=8, m=256, k=32)
    blocks = w["fd"]
    r = 40
    u, _ = oexact.top_left_basis(blocks, r)
    U = torch.tensor(u, dtype=torch.float32, device="cuda")
    got = csvd.tail_grad(U, [b.cuda() for b in blocks], 1.0)
    want = oexact.tail_grad(blocks, r)
    for g, wt in zip(got, want):
        np.testing.assert_allclose(_np(g), wt, atol=2e-5 * np.abs(wt).max())


def test_tail_energy_autograd_fd_full_size(csvd):
    """Config-5 check: 8 blocks 2048 x 256 from three latent subspaces with a
    large gap at r = 128; backward of the autograd function against central
    finite differences (h = 1e-3) of the FP64 oracle's exact tail."""
    w = synth.grad_c5(n_blocks=8)
    blocks = w["fd"]
    r = w["r"]
    s = oexact.singular_values(blocks)
    assert s[r - 1] / s[r] >= 1.5
    xs = [b.cuda().requires_grad_(True) for b in blocks]
    E = csvd.tail_energy(xs, r, working_rank=r + 32)
    E.backward()
    assert math.isclose(float(E.detach()), oexact.tail_sq(blocks, r), rel_tol=1e-3)
    rng = np.random.default_rng(0)
    h = 1e-3
    for _ in range(3):
        d = [rng.standard_normal(b.shape) for b in blocks]
        nrm = math.sqrt(sum(float(np.sum(x * x)) for x in d))
        d = [x / nrm for x in d]   # unit direction: h is a small step against the gap
        bp = [b.double().numpy() + h * x for b, x in zip(blocks, d)]
        bm = [b.double().numpy() - h * x for b, x in zip(blocks, d)]
        fd = (oexact.tail_sq(bp, r) - oexact.tail_sq(bm, r)) / (2 * h)
        an = sum(float(np.sum(_np(x.grad) * dd)) for x, dd in zip(xs, d))
        assert math.isclose(fd, an, rel_tol=1e-3), (fd, an)
    want = oexact.tail_grad(blocks, r)
    for x, wt in zip(xs, want):
        np.testing.assert_allclose(_np(x.grad), wt, atol=1e-3 * np.abs(wt).max())


# ------------------------------------------------------------------ errors
def test_argument_errors_return_status(csvd):
    import ctypes
    st = csvd.IncrSVD(16, 4)
    bad = csvd.Block(0, 4, 4, 0, 0)
    assert csvd.lib().csvd_incr_append(st.handle, ctypes.byref(bad)) == csvd.Status.ERR_ARG
    x = torch.zeros(16, 4, device="cuda")
    b = csvd.block(x)
    b.ld = 2
    assert csvd.lib().csvd_incr_append(st.handle, ctypes.byref(b)) == csvd.Status.ERR_ARG
    b = csvd.block(x)
    b.dtype = 9
    assert csvd.lib().csvd_incr_append(st.handle, ctypes.byref(b)) == csvd.Status.ERR_ARG
    st.append(x)   # still usable after rejected calls
    assert st.rank == 4


def test_residual_energy_and_top_basis_against_oracle(csvd):
    """csvd_tail_energy: ||(I - U U^T) A_j||^2 for a given orthonormal basis
    against the FP64 value, per block; csvd_top_basis: the refined basis
    spans the oracle's top-r subspace of the gapped collection (its tail
    energy equals the Eckart-Young tail)."""
    w = synth.grad_c5(n_blocks=8, m=512, k=64)
    blocks = w["fd"]
    r = 128
    u, _ = oexact.top_left_basis(blocks, r)
    U = torch.tensor(u, dtype=torch.float32, device="cuda")
    got = csvd.residual_energy(U, [b.cuda() for b in blocks])
    u32 = U.double().cpu().numpy()
    for j, b in enumerate(blocks):
        a = b.double().numpy()
        res = a - u32 @ (u32.T @ a)
        want = float(np.sum(res * res))
        _check_tail(got[j], want, float(np.sum(a * a)))
    Ug = csvd.top_basis([b.cuda() for b in blocks], r, r + 32, refine=2)
    assert Ug.shape == (512, r)
    tail = float(csvd.residual_energy(Ug, [b.cuda() for b in blocks]).sum())
    energy = sum(float((b.double() ** 2).sum()) for b in blocks)
    _check_tail(tail, oexact.tail_sq(blocks, r), energy)
