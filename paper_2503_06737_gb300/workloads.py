"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no hashing arithmetic: it only draws data.  The tests hand
the same arrays to the CUDA library and to the CPU oracle, and the bench
times the library on them.

The paper's real datasets (Sec. 6: Arcene, RNA-Seq, PEMS-SF, Gist) are not
available; these generators stand in for them with the shapes and value
distributions of the workload configurations:

* ``iid``       -- i.i.d. N(0, 1) rows (the 10,000 x 128 small case and the
                   4,000,000 x 512 dense precision sweep).
* ``gmm``       -- Gaussian mixture: component means ~ N(0, I), per-component
                   isotropic std ~ U[0.2, 1], equal weights (the Gist-shaped
                   1,000,000 x 960 set with 64 components, the 10,000,000 x 128
                   serving set with 1,024 components).
* ``csr_rows``  -- sparse non-negative rows: a fixed number of distinct,
                   uniformly placed columns per row (sorted), lognormal(0, 1)
                   values, each row scaled to unit L2 norm (200,000 x 20,000 at
                   1% density).
* ``noisy_queries`` -- database rows chosen by a seeded draw plus N(0, sigma^2)
                   noise per coordinate (sigma read as the standard deviation).

All draws use torch generators seeded explicitly, on the device the caller
names; the same (seed, device type) gives the same data.
"""
from __future__ import annotations

import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def iid(n: int, d: int, seed: int = 1234, device="cpu", dtype=torch.float32, chunk: int = 1 << 22):
    """n x d i.i.d. standard normal rows, stored in `dtype` (rounded once)."""
    g = _gen(seed, device)
    out = torch.empty((n, d), dtype=dtype, device=device)
    rows = max(1, chunk // max(d, 1))
    for s in range(0, n, rows):
        e = min(n, s + rows)
        out[s:e] = torch.randn((e - s, d), generator=g, device=device, dtype=torch.float32).to(dtype)
    return out


def gmm(n: int, d: int, components: int, seed: int = 1235, device="cpu", dtype=torch.float32,
        sigma_lo: float = 0.2, sigma_hi: float = 1.0, chunk: int = 1 << 22):
    """n x d rows from an equal-weight Gaussian mixture (means ~ N(0, I), std ~ U[lo, hi])."""
    g = _gen(seed, device)
    means = torch.randn((components, d), generator=g, device=device, dtype=torch.float32)
    sig = torch.rand((components,), generator=g, device=device, dtype=torch.float32)
    sig = sigma_lo + (sigma_hi - sigma_lo) * sig
    comp = torch.randint(0, components, (n,), generator=g, device=device)
    out = torch.empty((n, d), dtype=dtype, device=device)
    rows = max(1, chunk // max(d, 1))
    for s in range(0, n, rows):
        e = min(n, s + rows)
        c = comp[s:e]
        z = torch.randn((e - s, d), generator=g, device=device, dtype=torch.float32)
        out[s:e] = (means[c] + sig[c, None] * z).to(dtype)
    return out


def csr_rows(n: int, d: int, nnz_per_row: int, seed: int = 1236, device="cpu"):
    """CSR (rowptr int64 [n+1], cols int32 [n*k] ascending per row, vals float32 [n*k]).

    Columns: k distinct uniform positions per row (the first k of a random
    permutation score, i.e. top-k of i.i.d. uniform keys), sorted ascending.
    Values: lognormal(0, 1), then each row divided by its L2 norm.
    """
    g = _gen(seed, device)
    k = int(nnz_per_row)
    cols = torch.empty((n, k), dtype=torch.int32, device=device)
    vals = torch.empty((n, k), dtype=torch.float32, device=device)
    rows = max(1, (1 << 24) // max(d, 1))
    for s in range(0, n, rows):
        e = min(n, s + rows)
        u = torch.rand((e - s, d), generator=g, device=device)
        c = torch.topk(u, k, dim=1).indices.sort(dim=1).values
        cols[s:e] = c.to(torch.int32)
        v = torch.exp(torch.randn((e - s, k), generator=g, device=device))
        v = v / torch.linalg.vector_norm(v, dim=1, keepdim=True)
        vals[s:e] = v.to(torch.float32)
    rowptr = torch.arange(0, n + 1, device=device, dtype=torch.int64) * k
    return rowptr, cols.reshape(-1), vals.reshape(-1)


def noisy_queries(X: torch.Tensor, q: int, sigma: float, seed: int = 7):
    """q queries: seeded rows of X plus N(0, sigma^2) per coordinate, in X's dtype.
    Returns (Q, source_ids)."""
    g = _gen(seed, X.device)
    src = torch.randint(0, X.shape[0], (q,), generator=g, device=X.device)
    z = torch.randn((q, X.shape[1]), generator=g, device=X.device, dtype=torch.float32)
    Q = (X[src].to(torch.float32) + sigma * z).to(X.dtype)
    return Q, src


def fp8_rows(X: torch.Tensor):
    """Per-row-scaled FP8 E4M3 copy of X: scale_r = amax_r / 448 (1 when the row is
    zero), codes = round-to-nearest-even(x / scale_r).  Returns (codes uint8 view, scale f32)."""
    Xf = X.to(torch.float32)
    amax = Xf.abs().amax(dim=1)
    scale = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax))
    q = (Xf / scale[:, None]).to(torch.float8_e4m3fn)
    return q.view(torch.uint8), scale.to(torch.float32)


# The workload configurations, by what they are.
WORKLOADS = {
    "iid_10k_d128": dict(n=10_000, d=128, gen="iid", dtype="f32", m=16, L=10, w=4.0,
                         queries=100, query_sigma=0.1),
    "gmm64_1M_d960": dict(n=1_000_000, d=960, gen="gmm", components=64, dtype="f32", m=64,
                          L=50, w=4.0, hcs_dims=[8, 10, 12], hcs_mdims=[4, 4, 4]),
    "csr_200k_d20000": dict(n=200_000, d=20_000, gen="csr", nnz=200, m=256, L=20,
                            hcs_dims=[100, 200], hcs_mdims=[16, 16]),
    "iid_4M_d512_bf16": dict(n=4_000_000, d=512, gen="iid", dtype="bf16", m=32, L=64, w=4.0),
    "gmm1024_10M_d128_f16": dict(n=10_000_000, d=128, gen="gmm", components=1024, dtype="f16",
                                 m_hcs=16, m_cs=12, L=32, hcs_dims=[8, 16], hcs_mdims=[4, 4],
                                 query_sigma=0.05),
}


def torch_dtype(name: str):
    return {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[name]
