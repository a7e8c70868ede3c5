"""ctypes binding of the C ABI in include/lsh.h (argument marshalling only).

Every step of the hot path runs in liblsh_gb300.so; this module converts torch
tensors (device memory, streams) into the plain pointers and sizes the ABI
takes, and raises on a non-OK status.  It never computes a hash itself and has
no fallback: if the library is missing it raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblsh_gb300.so")

# Kinds and dtypes: the numbering of lsh_kind / lsh_dtype.
E2LSH, SRP, CS_E2LSH, HCS_E2LSH, CS_SRP, HCS_SRP, CSL_SRP = range(7)
KINDS = {"e2lsh": E2LSH, "srp": SRP, "cs_e2lsh": CS_E2LSH, "hcs_e2lsh": HCS_E2LSH,
         "cs_srp": CS_SRP, "hcs_srp": HCS_SRP, "csl_srp": CSL_SRP}
F32, BF16, F16, FP8_E4M3 = range(4)
_TORCH_DTYPE = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16, torch.uint8: FP8_E4M3,
                torch.float8_e4m3fn: FP8_E4M3}
STATUS = {0: "LSH_OK", 1: "LSH_EINVAL", 2: "LSH_ENOMEM", 3: "LSH_ECUDA", 4: "LSH_ETIMEOUT",
          5: "LSH_ENONFINITE", 6: "LSH_EUNSUPPORTED", 7: "LSH_ERANGE"}

MAX_MODES = 8


class LshError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class FamilyDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("d", ctypes.c_int32), ("m", ctypes.c_int32),
                ("L", ctypes.c_int32), ("N", ctypes.c_int32),
                ("dims", ctypes.c_int32 * MAX_MODES), ("mdims", ctypes.c_int32 * MAX_MODES),
                ("w", ctypes.c_double), ("seed", ctypes.c_uint64), ("compute", ctypes.c_int32),
                ("nnz_per_col", ctypes.c_int32)]


class Matrix(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("n", ctypes.c_int64), ("d", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("values", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("rowptr", ctypes.c_void_p), ("row_scale", ctypes.c_void_p)]


class HashStats(ctypes.Structure):
    _fields_ = [("n_entries", ctypes.c_int64), ("n_flagged", ctypes.c_int64),
                ("n_changed", ctypes.c_int64), ("n_nonfinite", ctypes.c_int64),
                ("n_overflow", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class QueryStats(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("n_candidates", ctypes.c_int64),
                ("n_unique", ctypes.c_int64), ("max_unique", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("slots", ctypes.c_int32), ("k", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("mem_budget", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed_requests", ctypes.c_int64), ("completed_queries", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("busy_s", ctypes.c_double), ("admitted_peak", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64), ("graph_captures", ctypes.c_int64)]

    def as_dict(self):
        return {k: (float(getattr(self, k)) if t is ctypes.c_double else int(getattr(self, k)))
                for k, t in self._fields_}


_lib = None

# (name, restype, argtypes) of every exported symbol of include/lsh.h
P = ctypes.c_void_p
SIGNATURES = [
    ("lsh_last_error", ctypes.c_char_p, []),
    ("lsh_version", ctypes.c_char_p, []),
    ("lsh_launch_count", ctypes.c_uint64, []),
    ("lsh_make_family", ctypes.c_int, [ctypes.POINTER(FamilyDesc), ctypes.POINTER(P)]),
    ("lsh_sample_family_tables", ctypes.c_int, [ctypes.POINTER(FamilyDesc), P, P, P, P, P, P]),
    ("lsh_family_describe", ctypes.c_int, [P, ctypes.POINTER(FamilyDesc)]),
    ("lsh_family_export", ctypes.c_int, [P, P, P, P, P, P, P]),
    ("lsh_family_status", ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    ("lsh_family_destroy", None, [P]),
    ("lsh_hash", ctypes.c_int, [P, ctypes.POINTER(Matrix), P, P, P, ctypes.POINTER(HashStats), P]),
    ("lsh_set_sketch_plan", ctypes.c_int, [ctypes.c_int32] * 6),
    ("lsh_set_sort_mode", ctypes.c_int, [ctypes.c_int32]),
    ("lsh_get_sketch_plan", ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int64, P]),
    ("lsh_build_index", ctypes.c_int, [P, ctypes.POINTER(Matrix), ctypes.c_int32, ctypes.POINTER(P), P]),
    ("lsh_index_rebuild", ctypes.c_int, [P, ctypes.POINTER(Matrix), P]),
    ("lsh_index_rebuild_host", ctypes.c_int, [P, ctypes.POINTER(Matrix), ctypes.c_int64, P]),
    ("lsh_index_info", ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64), P]),
    ("lsh_index_export", ctypes.c_int, [P, P, P, P, P]),
    ("lsh_query", ctypes.c_int, [P, ctypes.POINTER(Matrix), ctypes.c_int32, P, P,
                                 ctypes.POINTER(QueryStats), P]),
    ("lsh_index_destroy", None, [P]),
    ("lsh_index_save", ctypes.c_int, [P, ctypes.c_char_p]),
    ("lsh_index_load", ctypes.c_int, [P, ctypes.c_char_p, ctypes.POINTER(P)]),
    ("lsh_merge_topk", ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(P),
                                      ctypes.POINTER(P), P, P, P]),
    ("lsh_build_tables_static", ctypes.c_int, [P, ctypes.c_int64, ctypes.c_int32, P, P, P, P, P]),
    ("lsh_hasher_create", ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(P)]),
    ("lsh_hasher_run", ctypes.c_int, [P, P, ctypes.c_int64, P, ctypes.c_int64, P]),
    ("lsh_hasher_info", ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("lsh_hasher_destroy", None, [P]),
    ("lsh_server_create", ctypes.c_int, [P, ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]),
    ("lsh_server_submit", ctypes.c_int, [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    ("lsh_server_wait", ctypes.c_int, [P, ctypes.c_int64, P, P, ctypes.POINTER(ctypes.c_double)]),
    ("lsh_server_stats_get", ctypes.c_int, [P, ctypes.POINTER(ServerStats), ctypes.c_int32]),
    ("lsh_server_destroy", None, [P]),
]


def lib():
    """Load liblsh_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2503_06737_gb300.build` (there is no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def launch_count() -> int:
    return int(lib().lsh_launch_count())


def set_sketch_plan(rows_per_lane=0, row_groups=0, warps_per_table=0, tables_per_cta=0, entry_bytes=0,
                    split_bins=0):
    """Pin the dense-row sketch kernel's plan process-wide (all zeros: autotuned)."""
    _check(lib().lsh_set_sketch_plan(rows_per_lane, row_groups, warps_per_table, tables_per_cta, entry_bytes,
                                     split_bins))


def set_sort_mode(mode=0):
    """Sort of the table builds, process-wide: 0 automatic, 1 global LSD passes, 2 bucket sort."""
    _check(lib().lsh_set_sort_mode(int(mode)))


def _check(st: int):
    if st != 0:
        raise LshError(st, lib().lsh_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def dense_matrix(X: torch.Tensor, row_scale: torch.Tensor | None = None) -> Matrix:
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a 2-D tensor with unit column stride")
    if X.dtype not in _TORCH_DTYPE:
        raise ValueError(f"unsupported dtype {X.dtype}")
    mtx = Matrix()
    mtx.dtype = _TORCH_DTYPE[X.dtype]
    mtx.n, mtx.d = X.shape
    mtx.ld = X.stride(0) if X.shape[0] > 1 else X.shape[1]
    mtx.values = X.data_ptr() if X.numel() else None
    mtx.row_scale = None if row_scale is None else row_scale.data_ptr()
    return mtx


def csr_matrix(rowptr: torch.Tensor, col: torch.Tensor, values: torch.Tensor, d: int) -> Matrix:
    mtx = Matrix()
    mtx.dtype = F32
    mtx.n = rowptr.shape[0] - 1
    mtx.d = d
    mtx.ld = d
    mtx.values = values.data_ptr() if values.numel() else None
    mtx.col = col.data_ptr() if col.numel() else None
    mtx.rowptr = rowptr.data_ptr()
    return mtx


def make_desc(kind, d, m, L, w=4.0, seed=42, dims=None, mdims=None, compute=F32, l=1) -> FamilyDesc:
    desc = FamilyDesc()
    desc.kind = KINDS.get(kind, kind)
    desc.d, desc.m, desc.L = d, m, L
    if dims is None:
        dims, mdims = [d], [m]
    desc.N = len(dims)
    for k, (a, b) in enumerate(zip(dims, mdims)):
        desc.dims[k] = a
        desc.mdims[k] = b
    desc.w = float(w)
    desc.seed = int(seed)
    desc.compute = compute
    desc.nnz_per_col = int(l)
    return desc


def sample_family_tables(kind, d, m, L, w=4.0, seed=42, dims=None, mdims=None, compute=F32, l=1):
    """The library's host sampler alone (no device): dict of numpy tables."""
    import numpy as np
    desc = make_desc(kind, d, m, L, w, seed, dims, mdims, compute, l)
    dense = desc.kind in (E2LSH, SRP)
    dsum = 0 if dense else (d * max(1, l) if desc.kind == CSL_SRP else sum(desc.dims[k] for k in range(desc.N)))
    bins = np.empty((L, dsum), np.int32)
    signs = np.empty((L, dsum), np.int8)
    G = np.empty((d, m * L), np.float32) if dense else None
    b = np.empty((L, m), np.float64)
    ka = np.empty((L, m), np.uint32)
    kb = np.empty((L, m), np.uint32)
    p = lambda a: None if a is None or a.size == 0 else ctypes.c_void_p(a.ctypes.data)
    _check(lib().lsh_sample_family_tables(ctypes.byref(desc), p(bins), p(signs), p(G), p(b), p(ka), p(kb)))
    return dict(bins=bins, signs=signs, G=G, b=b, ka=ka, kb=kb)


class Family:
    """An LSH family drawn on the host and resident on the current device."""

    def __init__(self, kind, d, m, L, w=4.0, seed=42, dims=None, mdims=None, compute=F32, l=1):
        desc = make_desc(kind, d, m, L, w, seed, dims, mdims, compute, l)
        if dims is None:
            dims, mdims = [d], [m]
        h = ctypes.c_void_p()
        _check(lib().lsh_make_family(ctypes.byref(desc), ctypes.byref(h)))
        self.handle = h
        self.l = max(1, int(l))
        self.kind, self.d, self.m, self.L, self.w, self.seed = desc.kind, d, m, L, float(w), seed
        self.dims, self.mdims = list(dims), list(mdims)

    @property
    def is_srp(self):
        return self.kind in (SRP, CS_SRP, HCS_SRP, CSL_SRP)

    def export(self):
        """Host copies of the drawn tables (for parity checks)."""
        import numpy as np
        dsum = 0 if self.kind in (E2LSH, SRP) else (self.d * self.l if self.kind == CSL_SRP else sum(self.dims))
        bins = np.empty((self.L, dsum), np.int32)
        signs = np.empty((self.L, dsum), np.int8)
        G = np.empty((self.d, self.m * self.L), np.float32) if self.kind in (E2LSH, SRP) else None
        b = np.empty((self.L, self.m), np.float64)
        ka = np.empty((self.L, self.m), np.uint32)
        kb = np.empty((self.L, self.m), np.uint32)
        p = lambda a: None if a is None or a.size == 0 else ctypes.c_void_p(a.ctypes.data)
        _check(lib().lsh_family_export(self.handle, p(bins), p(signs), p(G), p(b), p(ka), p(kb)))
        return dict(bins=bins, signs=signs, G=G, b=b, ka=ka, kb=kb)

    def sketch_plan(self, n, dtype=torch.float32) -> dict:
        """The tile plan a dense-row hash of n rows would use now (pinned, tuned or default)."""
        import numpy as np
        v = np.zeros(6, np.int32)
        _check(lib().lsh_get_sketch_plan(self.handle, _TORCH_DTYPE[dtype], int(n), ctypes.c_void_p(v.ctypes.data)))
        keys = ("rows_per_lane", "row_groups", "warps_per_table", "tables_per_cta", "entry_bytes", "split_bins")
        return dict(zip(keys, (int(x) for x in v)))

    def status(self, clear=True) -> int:
        s = ctypes.c_int32()
        _check(lib().lsh_family_status(self.handle, ctypes.byref(s), int(clear)))
        return int(s.value)

    def code_shape(self, n):
        if self.is_srp:
            return (n, self.L, (self.m + 63) // 64), torch.int64
        return (n, self.L, self.m), torch.int32

    def hash(self, X=None, *, csr=None, codes=False, keys=True, proj=False, stats=False,
             row_scale=None, stream=None):
        """Hash a dense tensor X [n, d] (or csr=(rowptr, col, values)) on its device.
        Returns a dict with the requested outputs ('codes', 'keys', 'proj', 'stats')."""
        mtx = dense_matrix(X, row_scale) if csr is None else csr_matrix(*csr, d=self.d)
        n = int(mtx.n)
        dev = X.device if X is not None else csr[0].device
        out = {}
        if codes:
            shp, dt = self.code_shape(n)
            out["codes"] = torch.empty(shp, dtype=dt, device=dev)
        if keys:
            out["keys"] = torch.empty((self.L, n), dtype=torch.int64, device=dev)
        if proj:
            out["proj"] = torch.empty((n, self.L, self.m), dtype=torch.float32, device=dev)
        st = HashStats() if stats else None
        _check(lib().lsh_hash(self.handle, ctypes.byref(mtx), _ptr(out.get("codes")),
                              _ptr(out.get("keys")), _ptr(out.get("proj")),
                              ctypes.byref(st) if st is not None else None, _stream(stream)))
        if st is not None:
            out["stats"] = st.as_dict()
        return out

    def hash_into(self, mtx: Matrix, codes_ptr, keys_ptr, proj_ptr, stream=None, stats=None):
        """Raw-pointer form (the bench's end-to-end leg)."""
        _check(lib().lsh_hash(self.handle, ctypes.byref(mtx), codes_ptr, keys_ptr, proj_ptr,
                              ctypes.byref(stats) if stats is not None else None, _stream(stream)))

    def build_index(self, X=None, *, csr=None, keep_data=True, stream=None) -> "Index":
        mtx = dense_matrix(X) if csr is None else csr_matrix(*csr, d=self.d)
        h = ctypes.c_void_p()
        _check(lib().lsh_build_index(self.handle, ctypes.byref(mtx), int(bool(keep_data)),
                                     ctypes.byref(h), _stream(stream)))
        return Index(self, h)

    def close(self):
        if getattr(self, "handle", None):
            lib().lsh_family_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hasher:
    """Replayed hashing of uneven batches (keys only): one captured CUDA graph
    per batch-size bucket, replayed with the batch's pointer and row count."""

    def __init__(self, family: "Family", dtype=torch.float32, ld=None, max_rows=1 << 20):
        self.family = family
        self.dtype = dtype
        self.ld = int(ld if ld is not None else family.d)
        h = ctypes.c_void_p()
        _check(lib().lsh_hasher_create(family.handle, _TORCH_DTYPE[dtype], self.ld, int(max_rows), ctypes.byref(h)))
        self.handle = h

    def run(self, X: torch.Tensor, keys: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Keys [L, n] of the rows of X [n, d] (row stride ld); into keys if given ([L, >= n], int64)."""
        n = int(X.shape[0])
        if X.dtype != self.dtype or X.shape[1] != self.family.d or (n > 1 and X.stride(0) != self.ld) \
                or X.stride(1) != 1:
            raise ValueError("X must match the hasher's dtype, d and row stride")
        if keys is None:
            keys = torch.empty((self.family.L, n), dtype=torch.int64, device=X.device)
        _check(lib().lsh_hasher_run(self.handle, _ptr(X), n, _ptr(keys), int(keys.stride(0)), _stream(stream)))
        return keys

    def info(self):
        c, r = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().lsh_hasher_info(self.handle, ctypes.byref(c), ctypes.byref(r)))
        return dict(captures=int(c.value), replays=int(r.value))

    def close(self):
        if getattr(self, "handle", None):
            lib().lsh_hasher_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_index(family: "Family", path: str) -> "Index":
    """Load an index saved with Index.save; the family must match the file's."""
    h = ctypes.c_void_p()
    _check(lib().lsh_index_load(family.handle, str(path).encode(), ctypes.byref(h)))
    return Index(family, h)


def merge_topk(ids_list, dist_list, id_offsets):
    """Merge per-shard [q, k] top-k lists (numpy int32 / float32, ascending by
    (distance, local id)) into the global top-k by (distance, global id):
    returns (ids int64 [q, k], dist float32 [q, k]).  Host only."""
    import numpy as np
    S = len(ids_list)
    ids_c = [np.ascontiguousarray(x, np.int32) for x in ids_list]
    dst_c = [np.ascontiguousarray(x, np.float32) for x in dist_list]
    q, k = ids_c[0].shape
    offs = np.ascontiguousarray(id_offsets, np.int64)
    ip = (ctypes.c_void_p * S)(*[a.ctypes.data for a in ids_c])
    dp = (ctypes.c_void_p * S)(*[a.ctypes.data for a in dst_c])
    out_i = np.empty((q, k), np.int64)
    out_d = np.empty((q, k), np.float32)
    _check(lib().lsh_merge_topk(S, q, k, ip, dp, ctypes.c_void_p(offs.ctypes.data),
                                ctypes.c_void_p(out_i.ctypes.data), ctypes.c_void_p(out_d.ctypes.data)))
    return out_i, out_d


class Index:
    """The L hash tables over a batch of points (owns device memory)."""

    def __init__(self, family: Family, handle):
        self.family = family
        self.handle = handle

    def save(self, path: str):
        """Write the tables (and kept rows) to a file (lsh_index_save)."""
        _check(lib().lsh_index_save(self.handle, str(path).encode()))

    def rebuild(self, X, stream=None):
        mtx = dense_matrix(X)
        _check(lib().lsh_index_rebuild(self.handle, ctypes.byref(mtx), _stream(stream)))

    def rebuild_into(self, mtx: Matrix, stream=None):
        _check(lib().lsh_index_rebuild(self.handle, ctypes.byref(mtx), _stream(stream)))

    def rebuild_from_host(self, X_host, chunk_rows=0, stream=None):
        """Rebuild from a (pinned) host tensor: chunked copies overlap the hashing."""
        mtx = dense_matrix(X_host)
        _check(lib().lsh_index_rebuild_host(self.handle, ctypes.byref(mtx), int(chunk_rows), _stream(stream)))

    def info(self):
        import numpy as np
        n = ctypes.c_int64()
        nb = np.empty(self.family.L, np.int64)
        _check(lib().lsh_index_info(self.handle, ctypes.byref(n), ctypes.c_void_p(nb.ctypes.data)))
        return int(n.value), nb

    def export(self):
        import numpy as np
        n, _ = self.info()
        L = self.family.L
        ids = np.empty((L, n), np.uint32)
        ukeys = np.empty((L, max(n, 1)), np.uint64)
        offsets = np.empty((L, n + 1), np.uint32)
        nb = np.empty(L, np.int64)
        p = lambda a: ctypes.c_void_p(a.ctypes.data)
        _check(lib().lsh_index_export(self.handle, p(ids) if n else None, p(ukeys) if n else None,
                                      p(offsets), p(nb)))
        return dict(ids=ids, ukeys=ukeys, offsets=offsets, nb=nb)

    def query(self, Q, k=10, stats=False, stream=None):
        mtx = dense_matrix(Q)
        q = int(mtx.n)
        ids = torch.empty((q, k), dtype=torch.int32, device=Q.device)
        dist = torch.empty((q, k), dtype=torch.float32, device=Q.device)
        st = QueryStats() if stats else None
        _check(lib().lsh_query(self.handle, ctypes.byref(mtx), int(k), _ptr(ids), _ptr(dist),
                               ctypes.byref(st) if st is not None else None, _stream(stream)))
        out = {"ids": ids, "dist": dist}
        if st is not None:
            out["stats"] = st.as_dict()
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().lsh_index_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching serving loop over an index built with keep_data
    (lsh_server_* of include/lsh.h).  submit() takes host queries (numpy array
    or CPU tensor [q, d] of float32 / float16 / bfloat16) and returns a ticket;
    wait() returns (ids [q, k], dist [q, k], latency_ms) as numpy arrays."""

    def __init__(self, index: Index, max_batch=4096, slots=4, k=10, use_graphs=True, mem_budget=0):
        cfg = ServerConfig(max_batch, slots, k, int(bool(use_graphs)), int(mem_budget))
        h = ctypes.c_void_p()
        _check(lib().lsh_server_create(index.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle, self.index, self.k = h, index, k

    def submit(self, Q) -> int:
        import numpy as np
        if isinstance(Q, torch.Tensor):
            t = Q.detach().contiguous().cpu()
            dt = _TORCH_DTYPE[t.dtype]
            q = t.shape[0]
            ptr = ctypes.c_void_p(t.data_ptr())
            keep = t
        else:
            a = np.ascontiguousarray(Q)
            dt = {np.dtype(np.float32): F32, np.dtype(np.float16): F16}[a.dtype]
            q = a.shape[0]
            ptr = ctypes.c_void_p(a.ctypes.data)
            keep = a
        tk = ctypes.c_int64()
        _check(lib().lsh_server_submit(self.handle, ptr, dt, q, ctypes.byref(tk)))
        del keep
        self._q = getattr(self, "_q", {})
        self._q[int(tk.value)] = q
        return int(tk.value)

    def wait(self, ticket: int):
        import numpy as np
        q = self._q.pop(ticket)
        ids = np.empty((q, self.k), np.int32)
        dist = np.empty((q, self.k), np.float32)
        lat = ctypes.c_double()
        _check(lib().lsh_server_wait(self.handle, ticket, ctypes.c_void_p(ids.ctypes.data),
                                     ctypes.c_void_p(dist.ctypes.data), ctypes.byref(lat)))
        return ids, dist, float(lat.value)

    def stats(self, reset=False):
        st = ServerStats()
        _check(lib().lsh_server_stats_get(self.handle, ctypes.byref(st), int(bool(reset))))
        return st.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            lib().lsh_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
