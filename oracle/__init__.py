"""FP64 CPU oracle for the CS/HCS/dense LSH hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.  The arithmetic lives in ``lsh_oracle.c`` (plain C,
FP64, built with ``-ffp-contract=off``); this module compiles that file with
gcc and marshals numpy arrays into it.

What each function follows (paper: arXiv 2503.06737):

* ``family``        -- the random functions of Definitions 2-5 (h, s per mode,
                       Gaussian r for the dense baseline, offsets b), drawn with
                       SplitMix64 in the order documented in ``lsh_oracle.c``.
* ``hash_dense``    -- Definitions 2, 3, 12, 19, 25, 31 (projection summed in
                       FP64 in ascending coordinate order, then floor / sign).
* ``hash_csr``      -- the same on sparse rows (stored entries, ascending column).
* ``build_index``   -- the hash tables of the (m, tau)-amplified scheme of
                       Sec. 3.1: per table, points grouped by key, ordered by
                       (key, id).
* ``query``         -- probe, union of buckets, exact-distance top-k (Sec. 6).
* ``bruteforce_knn``-- exact ground truth for recall (Sec. 6).

Every function here is "pinned" by tests in ``tests/test_oracle_*.py`` against
closed forms, explicit matrices and brute force (see those files).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsh_oracle.c")
_LIB = os.path.join(_HERE, "liblsh_oracle.so")

# Kinds, in the numbering shared with the library's public header.
E2LSH, SRP, CS_E2LSH, HCS_E2LSH, CS_SRP, HCS_SRP, CSL_SRP = range(7)
KIND_NAMES = {"e2lsh": E2LSH, "srp": SRP, "cs_e2lsh": CS_E2LSH,
              "hcs_e2lsh": HCS_E2LSH, "cs_srp": CS_SRP, "hcs_srp": HCS_SRP, "csl_srp": CSL_SRP}
# Input dtypes: 0 f32, 1 bf16 (uint16 bits), 2 f16, 3 fp8 e4m3 (uint8 bits).
F32, BF16, F16, E4M3 = range(4)


def is_srp(kind: int) -> bool:
    return kind in (SRP, CS_SRP, HCS_SRP, CSL_SRP)


def is_dense(kind: int) -> bool:
    return kind in (E2LSH, SRP)


def compile_to(src: str, out: str) -> str:
    """gcc -O2 -ffp-contract=off -fopenmp: every FP64 operation one IEEE rounding, in source order."""
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC",
                           "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile lsh_oracle.c into liblsh_oracle.so next to it.  The tests that plant
    mistakes in a copy of the oracle point LSH_ORACLE_LIB at the mutant instead."""
    override = os.environ.get("LSH_ORACLE_LIB")
    if override:
        return override
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_to(_SRC, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int
U64 = ctypes.c_uint64
D = ctypes.c_double


def _declare(L):
    L.orc_mix64.restype = U64
    L.orc_mix64.argtypes = [U64]
    L.orc_splitmix_next.restype = U64
    L.orc_splitmix_next.argtypes = [ctypes.POINTER(U64)]
    L.orc_table_stream.restype = U64
    L.orc_table_stream.argtypes = [U64, I32]
    L.orc_family_tables.restype = None
    L.orc_family_tables.argtypes = [U64, I32, I32, P, P, D, P, P, P, P, P]
    L.orc_family_tables_l.restype = None
    L.orc_family_tables_l.argtypes = [U64, I32, I32, I32, I32, D, P, P, P, P, P]
    L.orc_dense_family.restype = None
    L.orc_dense_family.argtypes = [U64, I32, I32, I32, D, I32, P, P, P, P]
    for nm in ("orc_from_bf16", "orc_from_f16"):
        getattr(L, nm).restype = D
        getattr(L, nm).argtypes = [ctypes.c_uint16]
    L.orc_from_e4m3.restype = D
    L.orc_from_e4m3.argtypes = [ctypes.c_uint8]
    L.orc_round_e4m3.restype = D
    L.orc_round_e4m3.argtypes = [D]
    L.orc_cs_project.restype = None
    L.orc_cs_project.argtypes = [P, I32, P, P, I32, P]
    L.orc_hcs_project.restype = None
    L.orc_hcs_project.argtypes = [P, I32, I32, P, P, P, P, P]
    L.orc_dense_project.restype = None
    L.orc_dense_project.argtypes = [P, I32, P, I64, I64, I32, P]
    L.orc_e2lsh_code.restype = ctypes.c_int32
    L.orc_e2lsh_code.argtypes = [D, D, D, D, ctypes.POINTER(I32)]
    L.orc_srp_bit.restype = I32
    L.orc_srp_bit.argtypes = [D]
    L.orc_key.restype = U64
    L.orc_key.argtypes = [P, I32, I32, P, P]
    L.orc_hash_dense.restype = I32
    L.orc_hash_dense.argtypes = [P, P, I32, P, I64, I64, P, P, P]
    L.orc_hash_csr.restype = I32
    L.orc_hash_csr.argtypes = [P, I64, P, P, P, P, P, P]
    L.orc_build_index.restype = None
    L.orc_build_index.argtypes = [P, I64, I32, P, P, P, P]
    L.orc_query.restype = None
    L.orc_query.argtypes = [P, P, P, P, I64, I32, I32, P, I32, I64, P, I32, I64, I64,
                            P, I32, I32, P, P, P]
    L.orc_bruteforce_knn.restype = None
    L.orc_bruteforce_knn.argtypes = [I64, I32, P, I32, I64, P, I32, I64, I64, I32, I32, P, P]
    L.orc_distance.restype = D
    L.orc_distance.argtypes = [P, P, I32, I32]
    L.orc_num_threads.restype = I32
    L.orc_num_threads.argtypes = []


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


class _OrcFamily(ctypes.Structure):
    _fields_ = [("kind", I32), ("d", I32), ("m", I32), ("L", I32), ("N", I32),
                ("dims", ctypes.c_int32 * 8), ("mdims", ctypes.c_int32 * 8),
                ("w", D), ("bins", P), ("signs", P), ("G", P), ("b", P),
                ("ka", P), ("kb", P)]


@dataclass
class Family:
    """The oracle's own copy of an LSH family (all tables)."""
    kind: int
    d: int
    m: int
    L: int
    w: float
    seed: int
    dims: list
    mdims: list
    l: int = 1                        # CSSRP-L: nonzeros per column
    bins: np.ndarray | None = None    # [L, sum(dims)] int32
    signs: np.ndarray | None = None   # [L, sum(dims)] int8
    G: np.ndarray | None = None       # [d, m*L] float32 (dense kinds)
    b: np.ndarray = field(default=None)   # [L, m] float64
    ka: np.ndarray = field(default=None)  # [L, m] uint32
    kb: np.ndarray = field(default=None)  # [L, m] uint32

    @property
    def N(self) -> int:
        return self.l if self.kind == CSL_SRP else len(self.dims)

    def mode_tables(self, t: int):
        """Per-mode (h_k, s_k) of table t as lists of arrays."""
        out, o = [], 0
        for dk in self.dims:
            out.append((self.bins[t, o:o + dk], self.signs[t, o:o + dk]))
            o += dk
        return out

    def _c(self):
        f = _OrcFamily()
        f.kind, f.d, f.m, f.L, f.N = self.kind, self.d, self.m, self.L, self.N
        for k in range(len(self.dims)):
            f.dims[k] = self.dims[k]
            f.mdims[k] = self.mdims[k]
        f.w = self.w
        f.bins = None if self.bins is None else self.bins.ctypes.data
        f.signs = None if self.signs is None else self.signs.ctypes.data
        f.G = None if self.G is None else self.G.ctypes.data
        f.b, f.ka, f.kb = self.b.ctypes.data, self.ka.ctypes.data, self.kb.ctypes.data
        return f


def family(kind, d, m, L, w=4.0, seed=42, dims=None, mdims=None, compute=F32, l=1) -> Family:
    """Draw the family (Definitions 2-5) from `seed`.  CS kinds take dims=[d],
    mdims=[m]; HCS kinds take the mode sizes (prod(dims) >= d, prod(mdims) = m).
    Dense kinds: compute = BF16 (E4M3) rounds every Gaussian entry to bfloat16 (FP8 E4M3).
    CSSRP-L ("csl_srp", Table 1): l distinct bins per coordinate, tables [L, d*l]."""
    kind = KIND_NAMES.get(kind, kind)
    lb = lib()
    if kind == CSL_SRP:
        assert 1 <= l <= m
        bins = np.empty((L, d * l), np.int32)
        signs = np.empty((L, d * l), np.int8)
        b = np.empty((L, m), np.float64)
        ka = np.empty((L, m), np.uint32)
        kb = np.empty((L, m), np.uint32)
        lb.orc_family_tables_l(seed, L, d, m, l, w, _p(bins), _p(signs), _p(b), _p(ka), _p(kb))
        return Family(kind, d, m, L, float(w), seed, [d], [m], bins=bins, signs=signs, b=b, ka=ka, kb=kb, l=l)
    if is_dense(kind):
        G = np.empty((d, m * L), np.float32)
        b = np.empty((L, m), np.float64)
        ka = np.empty((L, m), np.uint32)
        kb = np.empty((L, m), np.uint32)
        lb.orc_dense_family(seed, L, d, m, w, int(compute), _p(G), _p(b), _p(ka), _p(kb))
        return Family(kind, d, m, L, float(w), seed, [d], [m], G=G, b=b, ka=ka, kb=kb)
    if kind in (CS_E2LSH, CS_SRP):
        dims, mdims = [d], [m]
    dims = [int(v) for v in dims]
    mdims = [int(v) for v in mdims]
    assert int(np.prod(mdims)) == m and int(np.prod(dims)) >= d and len(dims) == len(mdims)
    Dsum = sum(dims)
    bins = np.empty((L, Dsum), np.int32)
    signs = np.empty((L, Dsum), np.int8)
    b = np.empty((L, m), np.float64)
    ka = np.empty((L, m), np.uint32)
    kb = np.empty((L, m), np.uint32)
    da = np.asarray(dims, np.int32)
    ma = np.asarray(mdims, np.int32)
    lb.orc_family_tables(seed, L, len(dims), _p(da), _p(ma), w, _p(bins), _p(signs),
                         _p(b), _p(ka), _p(kb))
    return Family(kind, d, m, L, float(w), seed, dims, mdims, bins=bins, signs=signs,
                  b=b, ka=ka, kb=kb)


def _dtype_code(X: np.ndarray, dtype):
    if dtype is not None:
        return dtype
    if X.dtype == np.float32:
        return F32
    if X.dtype == np.float16:
        return F16
    raise ValueError("give dtype for raw-bit inputs (bf16 as uint16, e4m3 as uint8)")


def hash_dense(fam: Family, X: np.ndarray, dtype=None, row_scale=None, want_y=True,
               want_codes=True, want_keys=True):
    """Hash every row of X.  Returns (status, y [n,L,m] f64, codes [n,L,m] i32, keys [L,n] u64)."""
    X = np.ascontiguousarray(X)
    dt = _dtype_code(X, dtype)
    n = X.shape[0]
    ld = X.shape[1] if X.ndim == 2 else fam.d
    y = np.empty((n, fam.L, fam.m), np.float64) if want_y else None
    codes = np.empty((n, fam.L, fam.m), np.int32) if want_codes else None
    keys = np.empty((fam.L, n), np.uint64) if want_keys else None
    rs = None if row_scale is None else np.ascontiguousarray(row_scale, np.float32)
    f = fam._c()
    st = lib().orc_hash_dense(ctypes.byref(f), _p(X), dt, _p(rs), n, ld, _p(y), _p(codes), _p(keys))
    return st, y, codes, keys


def hash_csr(fam: Family, rowptr, cols, vals, want_y=True, want_codes=True, want_keys=True):
    """Hash CSR rows (int64 rowptr [n+1], int32 cols ascending per row, float32 vals)."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    cols = np.ascontiguousarray(cols, np.int32)
    vals = np.ascontiguousarray(vals, np.float32)
    n = rowptr.shape[0] - 1
    y = np.empty((n, fam.L, fam.m), np.float64) if want_y else None
    codes = np.empty((n, fam.L, fam.m), np.int32) if want_codes else None
    keys = np.empty((fam.L, n), np.uint64) if want_keys else None
    f = fam._c()
    st = lib().orc_hash_csr(ctypes.byref(f), n, _p(rowptr), _p(cols), _p(vals), _p(y),
                            _p(codes), _p(keys))
    return st, y, codes, keys


@dataclass
class Index:
    n: int
    L: int
    ids: np.ndarray      # [L, n] uint32
    ukeys: np.ndarray    # [L, n] uint64 (first nb[t] valid)
    offsets: np.ndarray  # [L, n+1] uint32 (first nb[t]+1 valid)
    nb: np.ndarray       # [L] int64

    def table(self, t):
        B = int(self.nb[t])
        return self.ids[t], self.ukeys[t, :B], self.offsets[t, :B + 1]


def build_index(keys: np.ndarray) -> Index:
    keys = np.ascontiguousarray(keys, np.uint64)
    L, n = keys.shape
    ids = np.empty((L, n), np.uint32)
    ukeys = np.zeros((L, max(n, 1)), np.uint64)
    offsets = np.zeros((L, n + 1), np.uint32)
    nb = np.zeros(L, np.int64)
    lib().orc_build_index(_p(keys), n, L, _p(ids), _p(ukeys), _p(offsets), _p(nb))
    return Index(n, L, ids, ukeys, offsets, nb)


def query(index: Index, d: int, X, Q, qkeys, k: int, metric: int, dtype=None, dtype_q=None):
    """Top-k over the union of the query's buckets.  Returns (ids [q,k], dist [q,k], ncand [q])."""
    X = np.ascontiguousarray(X)
    Q = np.ascontiguousarray(Q)
    qkeys = np.ascontiguousarray(qkeys, np.uint64)
    q = Q.shape[0]
    out_ids = np.empty((q, k), np.int32)
    out_dist = np.empty((q, k), np.float64)
    ncand = np.empty(q, np.int64)
    lib().orc_query(_p(index.ids), _p(index.ukeys), _p(index.offsets), _p(index.nb),
                    index.n, index.L, d, _p(X), _dtype_code(X, dtype), X.shape[1],
                    _p(Q), _dtype_code(Q, dtype_q), Q.shape[1], q, _p(qkeys), k, metric,
                    _p(out_ids), _p(out_dist), _p(ncand))
    return out_ids, out_dist, ncand


def bruteforce_knn(X, Q, k: int, metric: int, dtype=None, dtype_q=None):
    X = np.ascontiguousarray(X)
    Q = np.ascontiguousarray(Q)
    q = Q.shape[0]
    out_ids = np.empty((q, k), np.int32)
    out_dist = np.empty((q, k), np.float64)
    lib().orc_bruteforce_knn(X.shape[0], X.shape[1], _p(X), _dtype_code(X, dtype), X.shape[1],
                             _p(Q), _dtype_code(Q, dtype_q), Q.shape[1], q, k, metric,
                             _p(out_ids), _p(out_dist))
    return out_ids, out_dist


def cs_project(x, h, s, m):
    x = np.ascontiguousarray(x, np.float64)
    h = np.ascontiguousarray(h, np.int32)
    s = np.ascontiguousarray(s, np.int8)
    y = np.empty(m, np.float64)
    lib().orc_cs_project(_p(x), x.shape[0], _p(h), _p(s), m, _p(y))
    return y


def hcs_project(x, dims, mdims, hk, sk):
    """hk, sk: per-mode tables concatenated (or a list of per-mode arrays)."""
    x = np.ascontiguousarray(x, np.float64)
    if isinstance(hk, (list, tuple)):
        hk = np.concatenate(hk)
        sk = np.concatenate(sk)
    hk = np.ascontiguousarray(hk, np.int32)
    sk = np.ascontiguousarray(sk, np.int8)
    da = np.asarray(dims, np.int32)
    ma = np.asarray(mdims, np.int32)
    y = np.empty(int(np.prod(mdims)), np.float64)
    lib().orc_hcs_project(_p(x), x.shape[0], len(dims), _p(da), _p(ma), _p(hk), _p(sk), _p(y))
    return y


def e2lsh_code(y: float, scale: float, b: float, w: float):
    err = I32(0)
    c = lib().orc_e2lsh_code(float(y), float(scale), float(b), float(w), ctypes.byref(err))
    return int(c), int(err.value)


def srp_bit(y: float) -> int:
    return int(lib().orc_srp_bit(float(y)))


def key(codes, is_srp_kind: bool, ka, kb) -> int:
    c = np.ascontiguousarray(codes, np.int32)
    ka = np.ascontiguousarray(ka, np.uint32)
    kb = np.ascontiguousarray(kb, np.uint32)
    return int(lib().orc_key(_p(c), c.shape[0], int(is_srp_kind), _p(ka), _p(kb)))


def splitmix_stream(seed: int, t: int, count: int):
    st = U64(lib().orc_table_stream(seed, t))
    return [int(lib().orc_splitmix_next(ctypes.byref(st))) for _ in range(count)]


def mix64(z: int) -> int:
    return int(lib().orc_mix64(z))


def from_bf16(h): return float(lib().orc_from_bf16(int(h)))
def from_f16(h): return float(lib().orc_from_f16(int(h)))
def from_e4m3(q): return float(lib().orc_from_e4m3(int(q)))


def round_e4m3(v) -> float:
    """The nearest FP8 E4M3 value (ties to even, saturating at 448)."""
    return float(lib().orc_round_e4m3(float(v)))


def num_threads() -> int:
    return int(lib().orc_num_threads())
