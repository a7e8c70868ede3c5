"""Shared helpers of the GPU parity tests: run the CUDA library (through the C
ABI) and the FP64 oracle on the same seeded inputs and compare."""
import numpy as np
import torch

import oracle
from paper_2503_06737_gb300 import lsh

ORACLE_DTYPE = {torch.float32: oracle.F32, torch.bfloat16: oracle.BF16, torch.float16: oracle.F16}


def to_oracle(X: torch.Tensor):
    """Host copy of X as the oracle reads it (raw bits for 16-bit types)."""
    Xc = X.detach().cpu().contiguous()
    if Xc.dtype == torch.float32:
        return Xc.numpy(), oracle.F32
    return Xc.view(torch.int16).numpy().view(np.uint16), ORACLE_DTYPE[Xc.dtype]


def unpack_bits(words: np.ndarray, m: int) -> np.ndarray:
    """SRP codes [n, L, words] uint64 -> [n, L, m] int32 bits (bit l of word l // 64)."""
    w = words.view(np.uint64)
    l = np.arange(m)
    return ((w[..., l // 64] >> (l % 64).astype(np.uint64)) & np.uint64(1)).astype(np.int32)


def proj_tolerance(Xh64: np.ndarray, m: int, dense: bool = False):
    """Per-row scale for the projection check: 1e-5 relative to max(|y|, s), where s
    is the typical size of a projection: ||x|| / sqrt(m) for a sketch bin (Theorems
    13, 20), ||x|| for a dense Gaussian projection."""
    nrm = np.linalg.norm(Xh64, axis=1)
    return nrm if dense else nrm / np.sqrt(m)


def compare_hash(fam_args: dict, X: torch.Tensor, rows=None, check_proj=True):
    """Hash X on the GPU and the selected rows with the oracle; assert bit-exact
    codes and keys, projections within 1e-5 relative; return (gpu stats, max rel err)."""
    fam = lsh.Family(**fam_args)
    out = fam.hash(X, codes=True, keys=True, proj=check_proj, stats=True)
    torch.cuda.synchronize()
    n = X.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows)
    Xs = X[torch.as_tensor(rows, device=X.device)] if len(rows) != n else X
    Xh, dt = to_oracle(Xs)
    ofam = oracle.family(fam_args["kind"], fam_args["d"], fam_args["m"], fam_args["L"],
                         w=fam_args.get("w", 4.0), seed=fam_args.get("seed", 42),
                         dims=fam_args.get("dims"), mdims=fam_args.get("mdims"),
                         compute=fam_args.get("compute", 0), l=fam_args.get("l", 1))
    st, y, codes, keys = oracle.hash_dense(ofam, Xh, dtype=dt)
    assert st == 0
    m = fam_args["m"]
    rt = torch.as_tensor(rows, device=X.device, dtype=torch.long)
    gk = out["keys"][:, rt].cpu().numpy().view(np.uint64)
    gc = out["codes"][rt].cpu().numpy()
    if fam.is_srp:
        gc = unpack_bits(gc, m)
    assert np.array_equal(gc, codes), f"codes differ at {np.argwhere(gc != codes)[:5]}"
    assert np.array_equal(gk, keys), f"keys differ at {np.argwhere(gk != keys)[:5]}"
    rel = 0.0
    if check_proj:
        gp = out["proj"][rt].cpu().numpy().astype(np.float64)
        X64 = Xs.detach().cpu().to(torch.float64).numpy()
        dense = fam_args["kind"] in ("e2lsh", "srp")
        scale = np.maximum(np.abs(y), proj_tolerance(X64, m, dense)[:, None, None])
        err = np.abs(gp - y)
        assert (err[scale == 0] == 0).all()  # an all-zero row projects to exact zeros
        rel = float(np.max(err[scale > 0] / scale[scale > 0])) if (scale > 0).any() else 0.0
        assert rel <= 1e-5, rel
    fam.close()
    return out["stats"], rel


def oracle_keys(fam_args: dict, X: torch.Tensor):
    """Keys [L, n] of the FP64 oracle for the rows of X."""
    Xh, dt = to_oracle(X)
    ofam = oracle.family(fam_args["kind"], fam_args["d"], fam_args["m"], fam_args["L"],
                         w=fam_args.get("w", 4.0), seed=fam_args.get("seed", 42),
                         dims=fam_args.get("dims"), mdims=fam_args.get("mdims"),
                         compute=fam_args.get("compute", 0), l=fam_args.get("l", 1))
    st, _, _, keys = oracle.hash_dense(ofam, Xh, dtype=dt, want_y=False, want_codes=False)
    assert st == 0
    return keys


def compare_keys_only(fam_args: dict, X: torch.Tensor):
    """Hash X for keys only (the lean kernel instantiation) and compare with the oracle."""
    fam = lsh.Family(**fam_args)
    out = fam.hash(X, keys=True)
    torch.cuda.synchronize()
    gk = out["keys"].cpu().numpy().view(np.uint64)
    fam.close()
    keys = oracle_keys(fam_args, X)
    assert np.array_equal(gk, keys), f"keys differ at {np.argwhere(gk != keys)[:5]}"
