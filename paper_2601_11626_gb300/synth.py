"""Seeded synthetic block collections shaped like the paper's workloads.

This module only draws random numbers and lays them out in memory; it holds
none of the method's arithmetic (no projections, residuals, SVDs or error
formulas).  Both the CUDA path and the CPU oracle receive the tensors it
returns, so parity tests compare the two on identical inputs.

Every block is produced by its own generator seeded from (collection seed,
block index), so any subset of a large collection can be regenerated alone.

Collections (m = common row count, blocks are row-major m x k float32):

* ``latent_mixture`` -- A_j = Q_{c(j)} D G_j + w_j Q_{c'(j)} D G'_j + s N_j with
  Haar-orthonormal latent bases Q_c (m x d), a fixed latent spectrum D, Gaussian
  coefficient matrices G, a mixing weight w_j ~ U[0, w_max] with a second
  subspace c' != c, and i.i.d. Gaussian noise of standard deviation s.
* ``small_c1`` / ``mid_c2`` / ``scoring_c4`` / ``grad_c5`` -- the five workload
  recipes built on it (the 4096x4096 bf16 weight-collection recipe is
  ``weights_c3``).

The paper's own datasets (Section 4, dataset table) are not available; these
mixtures stand in for them with the same block shapes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

__all__ = [
    "Collection", "latent_bases", "latent_mixture", "small_c1", "mid_c2",
    "scoring_c4", "grad_c5", "weights_c3", "random_blocks", "pack_blocks",
]


def _gen(seed: int, *idx: int, device="cpu") -> torch.Generator:
    """Independent generator for (seed, idx...) -- a fixed 64-bit mix."""
    h = (seed * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    for i in idx:
        h ^= (i + 0x632BE59BD9B4E019 + ((h << 6) & 0xFFFFFFFFFFFFFFFF) + (h >> 2))
        h &= 0xFFFFFFFFFFFFFFFF
    g = torch.Generator(device=device)
    g.manual_seed(h & 0x7FFFFFFFFFFFFFFF)
    return g


def latent_bases(m: int, d: int, count: int, seed: int) -> list[torch.Tensor]:
    """``count`` Haar-distributed m x d orthonormal bases (QR of a Gaussian,
    column signs fixed by the R diagonal), float64 on the CPU."""
    out = []
    for c in range(count):
        g = _gen(seed, 1_000_003, c)
        z = torch.randn(m, d, generator=g, dtype=torch.float64)
        q, rr = torch.linalg.qr(z)
        q = q * torch.sign(torch.diagonal(rr)).unsqueeze(0)
        out.append(q)
    return out


@dataclass
class Collection:
    """A list of row-major float blocks sharing the row count ``m``."""
    m: int
    blocks: list
    latent: list = field(default_factory=list)   # latent subspace per block
    meta: dict = field(default_factory=dict)

    @property
    def widths(self):
        return [int(b.shape[1]) for b in self.blocks]


def latent_mixture(m, widths, bases, spectrum, noise, seed, *, assign=None,
                   w_max=0.0, device="cpu", dtype=torch.float32, ld_align=1,
                   index_offset=0, pool=None):
    """Draw one block per entry of ``widths`` (see module docstring).

    ``assign[j]`` is the primary latent subspace of block j (default j mod
    len(bases)).  When ``ld_align`` > 1 the blocks are views into one pooled
    allocation whose rows are padded to a multiple of ``ld_align`` elements
    (padding is zero)."""
    nb = len(bases)
    d = bases[0].shape[1]
    dvec = torch.as_tensor(spectrum, dtype=torch.float64)
    assert dvec.numel() == d
    bases_dev = [b.to(device=device, dtype=torch.float32) for b in bases]
    if assign is None:
        assign = [j % nb for j in range(len(widths))]
    lds = [((k + ld_align - 1) // ld_align) * ld_align for k in widths]
    if pool is None and ld_align > 1:
        total = sum(m * ld for ld in lds)
        pool = torch.zeros(total, device=device, dtype=dtype)
    blocks, off = [], 0
    latent = []
    for j, k in enumerate(widths):
        jj = j + index_offset
        g = _gen(seed, jj, device=device)
        c = assign[j]
        coeff = torch.randn(d, k, generator=g, device=device, dtype=torch.float32)
        coeff = coeff * dvec.to(device=device, dtype=torch.float32).unsqueeze(1)
        a = bases_dev[c] @ coeff
        if w_max > 0 and nb > 1:
            gw = _gen(seed, jj, 7, device="cpu")
            w = float(torch.rand((), generator=gw, dtype=torch.float64)) * w_max
            c2 = int(torch.randint(0, nb - 1, (), generator=gw))
            c2 = c2 + 1 if c2 >= c else c2
            coeff2 = torch.randn(d, k, generator=g, device=device, dtype=torch.float32)
            coeff2 = coeff2 * dvec.to(device=device, dtype=torch.float32).unsqueeze(1)
            a = a + w * (bases_dev[c2] @ coeff2)
        if noise > 0:
            a = a + noise * torch.randn(m, k, generator=g, device=device, dtype=torch.float32)
        a = a.to(dtype)
        if pool is not None:
            ld = lds[j]
            view = pool[off:off + m * ld].view(m, ld)[:, :k]
            view.copy_(a)
            blocks.append(view)
            off += m * ld
        else:
            blocks.append(a.contiguous())
        latent.append(c)
    return blocks, latent, pool


def small_c1(seed=0, device="cpu") -> Collection:
    """16 blocks 256x64: A_j = Q_{j mod 4} diag(2^{-i/2}) G_j + 1e-3 N_j with
    four 256x8 latent bases; rank 16, tolerance 0.05."""
    m, d = 256, 8
    bases = latent_bases(m, d, 4, seed)
    spec = [2.0 ** (-i / 2.0) for i in range(1, d + 1)]
    blocks, latent, _ = latent_mixture(m, [64] * 16, bases, spec, 1e-3, seed, device=device)
    return Collection(m, blocks, latent, dict(name="c1", r=16, eps=0.05))


def mid_c2(seed=0, device="cpu", n_blocks=256) -> Collection:
    """256 blocks 1024x128 from 16 latent 1024x32 subspaces, spectrum 0.9^i,
    second-subspace weight U[0,0.3], noise 1e-2; rank 64."""
    m, d = 1024, 32
    bases = latent_bases(m, d, 16, seed)
    spec = [0.9 ** i for i in range(1, d + 1)]
    blocks, latent, _ = latent_mixture(m, [128] * n_blocks, bases, spec, 1e-2, seed,
                                       w_max=0.3, device=device)
    return Collection(m, blocks, latent, dict(name="c2", r=64, eps=(0.02, 0.05, 0.1)))


def _widths(n, lo, hi, seed, tag):
    g = _gen(seed, tag)
    return [int(x) for x in torch.randint(lo, hi + 1, (n,), generator=g)]


def scoring_c4(r=64, seed=0, device="cpu", n_states=64, appends=8, per_state=64,
               m=2048, k_lo=16, k_hi=512, ld_align=8):
    """Batched merge scoring: ``n_states`` cluster states (state s is built
    from ``appends`` blocks of latent subspace s) and ``n_states*per_state``
    candidate blocks (candidate i is scored against state i // per_state and
    drawn from latent subspace i mod n_states).  Widths are i.i.d. uniform
    integers in [k_lo, k_hi]; blocks as in the mid-size recipe with
    ``n_states`` latent 2048x32 subspaces.  Candidate rows are padded to a
    multiple of ``ld_align`` floats inside one pooled allocation."""
    d = 32
    bases = latent_bases(m, d, n_states, seed)
    spec = [0.9 ** i for i in range(1, d + 1)]
    n_c = n_states * per_state
    st_w = _widths(n_states * appends, k_lo, k_hi, seed, 11)
    st_assign = [s for s in range(n_states) for _ in range(appends)]
    st_blocks, _, st_pool = latent_mixture(m, st_w, bases, spec, 1e-2, seed + 1,
                                           assign=st_assign, w_max=0.3, device=device,
                                           ld_align=ld_align)
    c_w = _widths(n_c, k_lo, k_hi, seed, 12)
    c_assign = [i % n_states for i in range(n_c)]
    c_blocks, _, c_pool = latent_mixture(m, c_w, bases, spec, 1e-2, seed + 2,
                                         assign=c_assign, w_max=0.3, device=device,
                                         ld_align=ld_align)
    states = [st_blocks[s * appends:(s + 1) * appends] for s in range(n_states)]
    cand_state = [i // per_state for i in range(n_c)]
    return dict(m=m, r=r, states=states, candidates=c_blocks, cand_state=cand_state,
                cand_latent=c_assign, pools=(st_pool, c_pool), eps=0.05)


def scoring_k1(seed=0, device="cpu", n_states=256, per_state=256, m=768, r=32, build=64,
               d=24, decay=0.9, noise=5e-2, w_max=0.3, eps=0.2):
    """One-column merge scoring with the k = 1 dataset's shape (768-dim
    vectors, r = 32, eps = 0.2): ``n_states`` latent m x d subspaces with
    spectrum ``decay``^i; state s is built from one m x ``build`` block of
    subspace s; candidate j (row j of the returned n x m matrix ``Xt``) is
    a vector of subspace j mod n_states plus a second subspace with weight
    U[0, w_max] and Gaussian noise, scored against state j // per_state (rows
    of one state are adjacent).  Vectorised per subspace; same recipe as
    ``latent_mixture`` with k = 1."""
    bases = latent_bases(m, d, n_states, seed)
    B = torch.stack([b.to(torch.float32) for b in bases]).to(device)       # n_states x m x d
    spec = torch.tensor([decay ** i for i in range(d)], dtype=torch.float32, device=device)
    g = _gen(seed, 31, device=device)
    st_coef = torch.randn(n_states, d, build, generator=g, device=device) * spec[None, :, None]
    st_blocks = torch.bmm(B, st_coef)
    st_blocks += noise * torch.randn(st_blocks.shape, generator=g, device=device)
    n = n_states * per_state
    c1 = torch.arange(n, device=device) % n_states
    gc = _gen(seed, 32, device="cpu")
    c2 = (c1.cpu() + 1 + torch.randint(0, n_states - 1, (n,), generator=gc)) % n_states
    w = torch.rand(n, generator=gc) * w_max
    coef1 = torch.randn(n, d, generator=g, device=device) * spec
    coef2 = torch.randn(n, d, generator=g, device=device) * spec * w.to(device)[:, None]
    Xt = noise * torch.randn(n, m, generator=g, device=device)
    c2 = c2.to(device)
    for c in range(n_states):
        rows = (c1 == c).nonzero().squeeze(1)
        Xt[rows] += coef1[rows] @ B[c].T
        rows2 = (c2 == c).nonzero().squeeze(1)
        Xt[rows2] += coef2[rows2] @ B[c].T
    cand_state = [j // per_state for j in range(n)]
    return dict(m=m, r=r, eps=eps, states=[[st_blocks[s]] for s in range(n_states)], Xt=Xt,
                cand_state=cand_state, cand_latent=c1.tolist())


def grad_c5(seed=0, device="cpu", n_blocks=1024, m=2048, k=256, fd_blocks=8):
    """Blocks 2048x256 from 32 latent subspaces of dimension 48.  Each latent
    spectrum has a strong head (43 directions, 42 for every third subspace)
    and a weak tail scaled by 0.05, so that a collection of ``fd_blocks``
    consecutive blocks (three subspaces, 128 strong directions) has a large
    gap sigma_128/sigma_129; noise 1e-3.  Returns the full collection and the
    gap-checked sub-collection."""
    d, nsub = 48, 32
    bases = latent_bases(m, d, nsub, seed)
    latent = []
    strong = [43 if c % 3 != 2 else 42 for c in range(nsub)]
    specs = []
    for c in range(nsub):
        s = [0.97 ** i if i <= strong[c] else 0.05 * 0.97 ** i for i in range(1, d + 1)]
        specs.append(s)
    assign = [j % 3 if j < fd_blocks else (j % nsub) for j in range(n_blocks)]
    out = []
    for j in range(n_blocks):
        c = assign[j]
        b, _, _ = latent_mixture(m, [k], [bases[c]], specs[c], 1e-3, seed,
                                 assign=[0], device=device, index_offset=j)
        out.append(b[0])
        latent.append(c)
    return dict(m=m, r=128, blocks=out, latent=latent, fd=out[:fd_blocks], eps=0.05)


def weights_c3(seed=0, device="cpu", n_mats=128, m=4096, shared_rank=256,
               resid_frac=0.3):
    """Weight-matrix-shaped collection, bf16 storage: W_i = B C_i + E_i with a
    shared orthonormal m x ``shared_rank`` basis B, Gaussian C_i and a
    residual E_i = X diag(j^-0.5) Y^T from random orthogonal factors, scaled
    to ``resid_frac`` of the block energy."""
    bases = latent_bases(m, shared_rank, 1, seed)[0].to(device=device, dtype=torch.float32)
    out = []
    for i in range(n_mats):
        g = _gen(seed, 50_000 + i, device=device)
        c = torch.randn(shared_rank, m, generator=g, device=device)
        w = bases @ c
        x, _ = torch.linalg.qr(torch.randn(m, m, generator=g, device=device))
        y, _ = torch.linalg.qr(torch.randn(m, m, generator=g, device=device))
        s = torch.arange(1, m + 1, device=device, dtype=torch.float32) ** -0.5
        e = (x * s.unsqueeze(0)) @ y.T
        e = e * math.sqrt(resid_frac / (1 - resid_frac)) * (w.norm() / e.norm())
        out.append((w + e).to(torch.bfloat16))
    return dict(m=m, r=256, blocks=out)


def random_blocks(m, widths, seed=0, *, rank=None, decay=1.0, noise=0.0,
                  dtype=torch.float32, device="cpu"):
    """Small generic collections for tests: each block is a random product of
    rank ``rank`` (default full) with singular-value decay ``decay`` per index,
    plus optional Gaussian noise."""
    out = []
    for j, k in enumerate(widths):
        g = _gen(seed, 900 + j)
        rk = min(m, k) if rank is None else rank
        a = torch.randn(m, rk, generator=g, dtype=torch.float64)
        s = torch.tensor([decay ** i for i in range(rk)], dtype=torch.float64)
        b = torch.randn(rk, k, generator=g, dtype=torch.float64)
        x = (a * s.unsqueeze(0)) @ b
        if noise:
            x = x + noise * torch.randn(m, k, generator=g, dtype=torch.float64)
        out.append(x.to(dtype).to(device))
    return out


def pack_blocks(blocks, ld_align=8, device=None):
    """Copy blocks into one pooled allocation with rows padded to a multiple
    of ``ld_align`` elements; returns (views, pool)."""
    device = device or blocks[0].device
    m = blocks[0].shape[0]
    lds = [((b.shape[1] + ld_align - 1) // ld_align) * ld_align for b in blocks]
    pool = torch.zeros(sum(m * ld for ld in lds), device=device, dtype=blocks[0].dtype)
    views, off = [], 0
    for b, ld in zip(blocks, lds):
        v = pool[off:off + m * ld].view(m, ld)[:, :b.shape[1]]
        v.copy_(b)
        views.append(v)
        off += m * ld
    return views, pool
