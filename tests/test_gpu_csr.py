"""GPU parity of lsh_hash on CSR rows (CS/HCS x SRP/E2LSH) against the oracle.

Sparse rows are the dense vectors with zeros at unstored positions; the
oracle's CSR path is itself pinned to its dense path.  Cases: the 20,000-wide
1%-dense lognormal workload (HCS 100 x 200 -> 16 x 16, m = 256), HCS with
odd, unit and power-of-two mode sizes, empty rows,
single nonzeros, rows longer than a warp, E2LSH on sparse rows, rows with
unsorted or out-of-range columns (rejected per row), and the full 200,000-row
workload checked on sampled rows.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_06737_gb300 import lsh, workloads

from gpu_helpers import unpack_bits

pytestmark = pytest.mark.gpu


def _csr_case(n, d, nnz, seed):
    rowptr, cols, vals = workloads.csr_rows(n, d, nnz, seed=seed, device="cpu")
    return rowptr, cols, vals


def _compare(args, rowptr, cols, vals, rows=None):
    fam = lsh.Family(**args)
    dev = [t.cuda() for t in (rowptr, cols, vals)]
    out = fam.hash(csr=tuple(dev), codes=True, keys=True, proj=True, stats=True)
    torch.cuda.synchronize()
    n = rowptr.shape[0] - 1
    rows = np.arange(n) if rows is None else np.asarray(rows)
    rp = rowptr.numpy()
    sub_rp = np.concatenate([[0], np.cumsum(rp[rows + 1] - rp[rows])]).astype(np.int64)
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if len(rows) else np.zeros(0, np.int64)
    c = cols.numpy()[idx]
    v = vals.numpy()[idx]
    of = oracle.family(args["kind"], args["d"], args["m"], args["L"], w=args.get("w", 4.0),
                       seed=args.get("seed", 42), dims=args.get("dims"), mdims=args.get("mdims"))
    st, y, codes, keys = oracle.hash_csr(of, sub_rp, c, v)
    assert st == 0
    rt = torch.as_tensor(rows, device="cuda", dtype=torch.long)
    gk = out["keys"][:, rt].cpu().numpy().view(np.uint64)
    gc = out["codes"][rt].cpu().numpy()
    if fam.is_srp:
        gc = unpack_bits(gc, args["m"])
    assert np.array_equal(gc, codes)
    assert np.array_equal(gk, keys)
    gp = out["proj"][rt].cpu().numpy().astype(np.float64)
    row_ids = np.repeat(np.arange(len(rows)), np.diff(sub_rp))
    nrm = np.sqrt(np.bincount(row_ids, weights=v.astype(np.float64) ** 2, minlength=len(rows)))
    scale = np.maximum(np.abs(y), (nrm / np.sqrt(args["m"]))[:, None, None])
    err = np.abs(gp - y)
    assert (err[scale == 0] == 0).all()
    if (scale > 0).any():
        assert float(np.max(err[scale > 0] / scale[scale > 0])) <= 1e-5
    return out["stats"]


@pytest.mark.parametrize("kind,dims,mdims", [("cs_srp", None, None), ("hcs_srp", [100, 200], [16, 16]),
                                             ("cs_e2lsh", None, None), ("hcs_e2lsh", [100, 200], [16, 16])])
@pytest.mark.parametrize("L", [5, 8, 20])
def test_csr_parity(kind, dims, mdims, L):
    # L a multiple of 4: count-sketch entries (not staged: 20,000 x L x 2 B) come four tables per load
    rowptr, cols, vals = _csr_case(600, 20000, 200, seed=3)
    st = _compare(dict(kind=kind, d=20000, m=256, L=L, w=0.5, seed=9, dims=dims, mdims=mdims), rowptr, cols, vals)
    assert st["n_nonfinite"] == 0


@pytest.mark.parametrize("kind,d,L", [("cs_srp", 100, 6), ("cs_e2lsh", 3000, 12), ("hcs_srp", 20000, 8)])
def test_csr_staged_and_long_rows(kind, d, L):
    """Entries staged in shared memory (small d), rows longer than the 256
    nonzeros a warp holds in registers (the rest is read per table), and
    rows of one nonzero."""
    rng = np.random.default_rng(14)
    n = 200
    lens = rng.integers(0, min(d, 700), size=n)
    lens[:4] = [1, min(d, 257), 0, min(d, 700) - 1]
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    cols = np.concatenate([np.sort(rng.choice(d, size=k, replace=False)) for k in lens]).astype(np.int32)
    vals = rng.lognormal(size=int(rowptr[-1])).astype(np.float32)
    dims, mdims = ([100, 200], [4, 8]) if kind.startswith("hcs") else (None, None)
    _compare(dict(kind=kind, d=d, m=32, L=L, w=0.5, seed=15, dims=dims, mdims=mdims), torch.from_numpy(rowptr),
             torch.from_numpy(cols), torch.from_numpy(vals))


def test_csr_exact_zero_bins():
    """Bins whose terms cancel exactly (x and -x in one bin), bins of -0.0
    values only, and all-zero rows: codes and keys still match the oracle."""
    d, m, L = 64, 8, 4
    args = dict(kind="cs_srp", d=d, m=m, L=L, seed=3)
    tabs = lsh.sample_family_tables(**args)
    h, sg = tabs["bins"][0], tabs["signs"][0]
    rows, cols, vals = [0], [], []
    for l in range(m):  # row l: two same-sign members of bin l of table 0 with values v and -v
        mem = [j for j in range(d) if h[j] == l]
        same = [j for j in mem if sg[j] == sg[mem[0]]]
        if len(same) >= 2:
            cols += [same[0], same[1]]
            vals += [0.75, -0.75]
        rows.append(len(cols))
    cols += [3, 9, 20]
    vals += [-0.0, -0.0, -0.0]
    rows.append(len(cols))
    cols += [1, 2]
    vals += [0.0, 0.0]
    rows.append(len(cols))
    _compare(args, torch.tensor(rows, dtype=torch.int64), torch.tensor(cols, dtype=torch.int32),
             torch.tensor(vals, dtype=torch.float32))


@pytest.mark.parametrize("kind,dims,mdims", [("hcs_srp", [13, 17, 23], [2, 4, 2]), ("hcs_e2lsh", [1, 71, 71], [1, 4, 4]),
                                             ("hcs_srp", [2, 2500], [4, 64])])
def test_csr_hcs_mode_sizes(kind, dims, mdims):
    """HCS on sparse rows with three odd mode sizes, a mode of size 1, and a
    power-of-two mode beside a large one: the mode indices of a column come
    from multiply-high quotients, checked here against the oracle."""
    rowptr, cols, vals = _csr_case(300, 5000, 60, seed=11)
    m = int(np.prod(mdims))
    _compare(dict(kind=kind, d=5000, m=m, L=4, w=0.5, seed=12, dims=dims, mdims=mdims), rowptr, cols, vals)


@pytest.mark.parametrize("kind", ["cs_srp", "cs_e2lsh"])
def test_csr_ragged_rows(kind):
    rng = np.random.default_rng(4)
    d, n = 5000, 300
    lens = rng.integers(0, 120, size=n)
    lens[:5] = [0, 1, 0, 64, 119]
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    cols = np.concatenate([np.sort(rng.choice(d, size=k, replace=False)) for k in lens]).astype(np.int32)
    vals = rng.standard_normal(int(rowptr[-1])).astype(np.float32)
    _compare(dict(kind=kind, d=d, m=32, L=4, w=1.0, seed=5), torch.from_numpy(rowptr),
             torch.from_numpy(cols), torch.from_numpy(vals))


def test_csr_small_m_srp_words():
    rowptr, cols, vals = _csr_case(100, 3000, 30, seed=6)
    _compare(dict(kind="cs_srp", d=3000, m=20, L=3, seed=7), rowptr, cols, vals)
    _compare(dict(kind="cs_srp", d=3000, m=64, L=3, seed=7), rowptr, cols, vals)


def test_csr_invalid_rows_rejected():
    rowptr = torch.tensor([0, 3, 6, 8], dtype=torch.int64)
    cols = torch.tensor([1, 5, 9, 4, 2, 7, 0, 3000], dtype=torch.int32)  # row 1 unsorted, row 2 col >= d
    vals = torch.ones(8, dtype=torch.float32)
    fam = lsh.Family("cs_srp", 1000, 16, 3, seed=1)
    with pytest.raises(lsh.LshError):
        fam.hash(csr=(rowptr.cuda(), cols.cuda(), vals.cuda()), keys=True, stats=True)
    out = fam.hash(csr=(rowptr.cuda(), cols.cuda(), vals.cuda()), keys=True)
    k = out["keys"].cpu().numpy().view(np.uint64)
    assert (k[:, 1] == np.uint64(0xFFFFFFFFFFFFFFFF)).all() and (k[:, 2] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    assert fam.status() != 0


@pytest.mark.parametrize("kind,dims,mdims", [("cs_srp", None, None), ("hcs_srp", [100, 200], [16, 16])])
def test_csr_full_size_sampled(kind, dims, mdims):
    wl = workloads.WORKLOADS["csr_200k_d20000"]
    rowptr, cols, vals = workloads.csr_rows(wl["n"], wl["d"], wl["nnz"], seed=1236, device="cuda")
    args = dict(kind=kind, d=wl["d"], m=wl["m"], L=wl["L"], seed=42, dims=dims, mdims=mdims)
    fam = lsh.Family(**args)
    out = fam.hash(csr=(rowptr, cols, vals), codes=True, keys=True, stats=True)
    rows = np.sort(np.random.default_rng(3).choice(wl["n"], 1500, replace=False))
    rp = rowptr.cpu().numpy()
    c_all, v_all = cols.cpu().numpy(), vals.cpu().numpy()
    sub_rp = np.concatenate([[0], np.cumsum(rp[rows + 1] - rp[rows])]).astype(np.int64)
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    of = oracle.family(kind, wl["d"], wl["m"], wl["L"], seed=42, dims=dims, mdims=mdims)
    st, _, codes, keys = oracle.hash_csr(of, sub_rp, c_all[idx], v_all[idx], want_y=False)
    rt = torch.as_tensor(rows, device="cuda")
    assert np.array_equal(out["keys"][:, rt].cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(unpack_bits(out["codes"][rt].cpu().numpy(), wl["m"]), codes)
    assert out["stats"]["n_entries"] == wl["n"] * wl["L"] * wl["m"]
    ko = fam.hash(csr=(rowptr, cols, vals), keys=True)  # keys only, as the bench times it
    assert torch.equal(ko["keys"], out["keys"])
