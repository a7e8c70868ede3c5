"""Benchmark of the LSH indexing hot path on GB300 (one JSON line on rank 0).

Step = one pass of the whole indexing path over one batch: CS/HCS hashing of
all L tables (with the FP64 boundary recheck and key fold) -> per-table
stable sort of (key, id) (the bucket sort: one global radix pass, buckets
finished on chip) -> bucket segmentation, i.e. lsh_index_rebuild
on a resident batch.  Workload (default): 1,000,000 x 960 FP32 points from a
64-component Gaussian mixture (the Gist-shaped set), CS-E2LSH, m = 64, L = 50,
w = 4.  Inputs (3.84 GB) are larger than L2 (129 MB), so no flush is needed.

value  = points indexed per second over all ranks (weak scaling: each rank
         indexes its own batch; no data-path collective).
e2e    = the same through the public API with host buffers: pinned host X ->
         device, rebuild, device -> host read of the per-table bucket counts.
roofline = the dominant kernel (the CS/HCS hashing kernel) timed alone with
         CUDA events on its stream.
cpu_baseline = the FP64 oracle on a bounded sample of the same workload, on
         the host cores (rank 0, N = 1 only).

--impl reference runs that oracle as the reference arm (host cores only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

T_START = time.time()


def log(msg):
    print(f"[bench +{time.time() - T_START:7.1f}s] {msg}", file=sys.stderr, flush=True)


METRIC = "hashed pts/s & HBM roofline %, CS/HCS vs dense; serve QPS, p99 @recall10≥0.9"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.lines = []
        self.window = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))

    def mark(self):
        return time.time()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if not (t0 - 0.15 <= ts <= t1 + 0.15):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def shard_seed(rank: int) -> int:
    """Data seed of a rank's shard: every rank hashes its own rows (weak
    scaling; the points are independent, so no data-path exchange)."""
    return 1235 + rank


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (the job's time) via one all-reduce MAX."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(world: int, n_per_rank: int, ms: float) -> float:
    """Points per second of the whole job: all ranks' points over the job's time."""
    return world * n_per_rank / (ms / 1e3)


def _source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel_key: str, workload: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary,
    if it was taken on the current source of that kernel (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel_key]
    except Exception:
        return None
    if rec.get("workload") != workload:
        return None
    if rec.get("source_sha") != _source_sha(rec.get("sources", [])):
        return None
    return rec.get("dram_bytes_per_launch")


def _gpu_local_cpus(dev) -> set:
    """The CPUs of the host memory node attached to the GPU (its PCI device's
    local_cpulist in sysfs), within this process's CPU set; empty if unknown."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                lo, hi = part.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif part:
                cpus.add(int(part))
        return cpus & os.sched_getaffinity(0)
    except Exception:
        return set()


def _pinned_near_gpu(shape, dtype, dev):
    """A pinned host buffer whose pages come from the GPU's own host memory
    node: the calling thread runs on that node's CPUs while the buffer is
    allocated (the pages are placed where the allocating thread runs), then
    gets its CPU set back.  A buffer on the other node of a two-socket host
    crosses the socket link on every host-to-device copy."""
    import torch
    saved = os.sched_getaffinity(0)
    local = _gpu_local_cpus(dev)
    bind = bool(local) and local != saved
    try:
        if bind:
            os.sched_setaffinity(0, local)
        buf = torch.empty(shape, dtype=dtype, pin_memory=True)
        buf.zero_()
    finally:
        if bind:
            os.sched_setaffinity(0, saved)
    return buf, (f"pinned on the GPU's host node ({len(local)} local CPUs)" if bind else
                 "pinned (node placement left to the OS)")


def _workload(name, kind):
    from paper_2503_06737_gb300 import workloads
    wl = dict(workloads.WORKLOADS[name])
    hcs = kind.startswith("hcs")
    fam = dict(kind=kind, d=wl["d"], m=wl["m"], L=wl["L"], w=wl.get("w", 4.0), seed=42,
               dims=wl["hcs_dims"] if hcs else None, mdims=wl["hcs_mdims"] if hcs else None)
    return wl, fam


def _make_X(wl, seed, device):
    import torch
    from paper_2503_06737_gb300 import workloads
    dt = workloads.torch_dtype(wl.get("dtype", "f32"))
    if wl["gen"] == "gmm":
        return workloads.gmm(wl["n"], wl["d"], wl["components"], seed=seed, device=device, dtype=dt)
    return workloads.iid(wl["n"], wl["d"], seed=seed, device=device, dtype=dt)


def _oracle_setup(wl, fam_args, seed=1235):
    import numpy as np
    import torch

    import oracle
    from paper_2503_06737_gb300 import workloads
    of = oracle.family(fam_args["kind"], fam_args["d"], fam_args["m"], fam_args["L"], w=fam_args["w"],
                       seed=fam_args["seed"], dims=fam_args["dims"], mdims=fam_args["mdims"])
    dt = workloads.torch_dtype(wl.get("dtype", "f32"))

    def sample(rows):
        X = workloads.gmm(rows, wl["d"], wl["components"], seed=seed, device="cpu", dtype=dt) \
            if wl["gen"] == "gmm" else workloads.iid(rows, wl["d"], seed=seed, device="cpu", dtype=dt)
        Xc = X.contiguous()
        if Xc.dtype == torch.float32:
            return Xc.numpy(), oracle.F32
        return Xc.view(torch.int16).numpy().view(np.uint16), {torch.bfloat16: oracle.BF16,
                                                             torch.float16: oracle.F16}[Xc.dtype]

    def step(Xh, dtc):
        """One oracle step on a sample: FP64 hash of every table, then the index."""
        t = time.perf_counter()
        st, _, _, keys = oracle.hash_dense(of, Xh, dtype=dtc, want_y=False, want_codes=False)
        oracle.build_index(keys)
        return time.perf_counter() - t

    def calibrate(target_s):
        rows = 256
        Xh, dtc = sample(rows)
        t = step(Xh, dtc)
        rows = int(min(wl["n"], max(rows, rows * target_s / max(t, 1e-3))))
        return rows, sample(rows)

    return step, calibrate, oracle.num_threads()


def oracle_sample_rate(wl, fam_args, target_s=15.0):
    """Points/s of the oracle (hash + index) on a bounded sample, host cores."""
    step, calibrate, cores = _oracle_setup(wl, fam_args)
    rows, (Xh, dtc) = calibrate(target_s)
    t = step(Xh, dtc)
    return rows / t, rows, t, cores


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores; each
    step hashes and indexes a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, fam_args = _workload(args.workload, args.kind)
    step, calibrate, cores = _oracle_setup(wl, fam_args)
    rows, (Xh, dtc) = calibrate(max(0.5, 90.0 / (args.steps + args.warmup)))
    for _ in range(args.warmup):
        step(Xh, dtc)
    ts = [step(Xh, dtc) for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    rate = rows / t
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "kind": fam_args["kind"], "n_per_gpu": wl["n"], "d": wl["d"],
                   "m": fam_args["m"], "L": fam_args["L"], "sample_rows_per_step": rows},
        "cpu_baseline": {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows} rows of {args.workload} per step ({fam_args['kind']} hash + index)"},
        "e2e": {"value": rate, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def extra_variants(args, X, keys, peaks, alu_peak, e0, e1, stream):
    """Dense FP32 GEMM baseline at the same m*L, the CSR workload, and the small
    index + query workload (each timed with CUDA events on the launching stream)."""
    import torch
    from paper_2503_06737_gb300 import lsh, measure, workloads
    out = {}
    wl, fa = _workload(args.workload, "e2lsh")
    n, d, L, m = X.shape[0], X.shape[1], fa["L"], fa["m"]
    mtx = lsh.dense_matrix(X)
    fd = lsh.Family(**fa)
    fd.hash_into(mtx, None, lsh._ptr(keys), None)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        fd.hash_into(mtx, None, lsh._ptr(keys), None)
    e1.record(stream)
    torch.cuda.synchronize()
    dms = e0.elapsed_time(e1) / 3
    flops = 2.0 * n * d * m * L
    st = fd.hash(X[:65536], keys=True, stats=True)["stats"]
    out["dense_fp32_e2lsh"] = {"hash_ms": dms, "points_per_s": n / (dms / 1e3), "tflops": flops / (dms / 1e3) / 1e12,
                               "flagged_per_entry": st["n_flagged"] / max(1, st["n_entries"]),
                               "note": "FP32 SIMT GEMM x G (d x mL = %d x %d) + fused epilogue, same m*L" % (d, m * L)}
    fd.close()
    # the same dense baseline on the tensor cores: BF16 copy of the rows, BF16 G
    Xb = X.to(torch.bfloat16)
    mtxb = lsh.dense_matrix(Xb)
    fb = lsh.Family(**dict(fa, compute=lsh.BF16))
    fb.hash_into(mtxb, None, lsh._ptr(keys), None)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        fb.hash_into(mtxb, None, lsh._ptr(keys), None)
    e1.record(stream)
    torch.cuda.synchronize()
    bms = e0.elapsed_time(e1) / 3
    st = fb.hash(Xb[:65536], keys=True, stats=True)["stats"]
    out["dense_bf16_tcgen05_e2lsh"] = {
        "hash_ms": bms, "points_per_s": n / (bms / 1e3), "tflops": flops / (bms / 1e3) / 1e12,
        "tensor_frac": flops / (bms / 1e3) / 1e12 / peaks.get("bf16_tflops", 1900.0),
        "flagged_per_entry": st["n_flagged"] / max(1, st["n_entries"]),
        "note": "tcgen05 BF16 x BF16 -> FP32 + exact recheck; BF16 copy of the rows (an input rounding the "
                "CS/HCS paths do not make), same m*L"}
    fb.close()
    del Xb, mtxb
    # CSR workload: 200,000 x 20,000 at 1%, m = 256, L = 20
    cw = workloads.WORKLOADS["csr_200k_d20000"]
    rowptr, cols, vals = workloads.csr_rows(cw["n"], cw["d"], cw["nnz"], seed=1236, device=X.device)
    ck = torch.empty((cw["L"], cw["n"]), dtype=torch.int64, device=X.device)
    cm = lsh.csr_matrix(rowptr, cols, vals, cw["d"])
    for kind, dims, mdims in (("cs_srp", None, None), ("hcs_srp", cw["hcs_dims"], cw["hcs_mdims"])):
        fc = lsh.Family(kind, cw["d"], cw["m"], cw["L"], seed=42, dims=dims, mdims=mdims)
        fc.hash_into(cm, None, lsh._ptr(ck), None)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            fc.hash_into(cm, None, lsh._ptr(ck), None)
        e1.record(stream)
        torch.cuda.synchronize()
        cms = e0.elapsed_time(e1) / 10
        cbytes = float(vals.numel() * 4 + cols.numel() * 4 + rowptr.numel() * 8 + ck.numel() * 8)
        out["csr_200k_d20000_" + kind] = {"hash_ms": cms, "points_per_s": cw["n"] / (cms / 1e3),
                                          "hbm_frac": cbytes / (cms / 1e3) / 1e9 / peaks["hbm_gbs"],
                                          "adds_per_s": float(vals.numel()) * cw["L"] / (cms / 1e3)}
        fc.close()
    del rowptr, cols, vals, ck
    # small workload: 10,000 x 128, CS-E2LSH m = 16, L = 10: index build + 100 queries
    sw = workloads.WORKLOADS["iid_10k_d128"]
    Xs = workloads.iid(sw["n"], sw["d"], seed=1234, device=X.device)
    Qs, _ = workloads.noisy_queries(Xs, sw["queries"], sw["query_sigma"], seed=7)
    fs = lsh.Family("cs_e2lsh", sw["d"], sw["m"], sw["L"], w=sw["w"], seed=42)
    idx = fs.build_index(Xs, keep_data=True)
    ms_b = lsh.dense_matrix(Xs)
    for _ in range(3):
        idx.rebuild_into(ms_b)
        idx.query(Qs, k=10)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(20):
        idx.rebuild_into(ms_b)
    e1.record(stream)
    torch.cuda.synchronize()
    bms = e0.elapsed_time(e1) / 20
    e0.record(stream)
    for _ in range(20):
        idx.query(Qs, k=10)
    e1.record(stream)
    torch.cuda.synchronize()
    qms = e0.elapsed_time(e1) / 20
    out["iid_10k_d128_build_and_query"] = {"build_us": bms * 1e3, "query_100_us": qms * 1e3,
                                           "qps": sw["queries"] / (qms / 1e3)}
    idx.close()
    fs.close()
    # the same small workload with the other families of the configuration:
    # CS-SRP and the dense E2LSH / SRP baselines (FP32 SIMT), build + 100 queries
    truth, _ = measure.exact_knn(Xs, Qs, 10)
    truth = truth.cpu().numpy()
    for kind in ("cs_e2lsh", "cs_srp", "e2lsh", "srp"):
        fk = lsh.Family(kind, sw["d"], sw["m"], sw["L"], w=sw["w"], seed=42)
        ik = fk.build_index(Xs, keep_data=True)
        for _ in range(3):
            ik.rebuild_into(ms_b)
            ik.query(Qs, k=10)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(20):
            ik.rebuild_into(ms_b)
        e1.record(stream)
        torch.cuda.synchronize()
        b2 = e0.elapsed_time(e1) / 20
        e0.record(stream)
        for _ in range(20):
            res = ik.query(Qs, k=10)
        e1.record(stream)
        torch.cuda.synchronize()
        q2 = e0.elapsed_time(e1) / 20
        out["iid_10k_d128_" + kind] = {"build_us": b2 * 1e3, "query_100_us": q2 * 1e3,
                                       "recall10": measure.recall_at_k(res["ids"].cpu().numpy(), truth)}
        ik.close()
        fk.close()
    del Xs, Qs
    log("small workload done; precision sweep")
    out["iid_4M_d512_bf16"] = precision_sweep(peaks, alu_peak, e0, e1, stream, X.device)
    return out


def uneven_batches(X, keys, e0, e1, stream, batches=200, seed=11):
    """Uneven hashing batches (row counts log-uniform in two ranges), keys
    only, CS-E2LSH m = 64, L = 50 on the headline rows: one lsh_hash call per
    batch against one lsh_hasher replay per batch (a captured CUDA graph per
    power-of-two size bucket).  Device time (CUDA events around the whole
    sequence) and host wall time per batch."""
    import math
    import numpy as np
    import torch
    from paper_2503_06737_gb300 import lsh
    d = X.shape[1]
    fam = lsh.Family("cs_e2lsh", d, 64, 50, w=4.0, seed=42)
    key_ld = keys.shape[1]
    rng = np.random.default_rng(seed)
    out = {"family": "cs_e2lsh m=64 L=50", "batches": batches}
    for lo, hi in ((64, 8192), (8192, 131072)):
        sizes = [int(math.exp(rng.uniform(math.log(lo), math.log(hi)))) for _ in range(batches)]
        mtx = [lsh.dense_matrix(X[:n]) for n in sizes]
        h = lsh.Hasher(fam, dtype=X.dtype, max_rows=hi)
        xp, kp = lsh._ptr(X), lsh._ptr(keys)
        st = lsh._stream(stream)

        def direct():
            for mt in mtx:
                fam.hash_into(mt, None, kp, None, stream=stream)

        def replay():
            for nb in sizes:
                lsh._check(lsh.lib().lsh_hasher_run(h.handle, xp, nb, kp, key_ld, st))

        row = {"rows": int(sum(sizes))}
        for name, fn in (("lsh_hash", direct), ("hasher_graphs", replay)):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            row[name] = {"device_ms": e0.elapsed_time(e1), "wall_ms": wall * 1e3,
                         "us_per_batch": wall * 1e6 / batches, "points_per_s": row["rows"] / wall}
        row["hasher_info"] = h.info()
        out[f"rows_{lo}_{hi}"] = row
        h.close()
    fam.close()
    return out


def precision_sweep(peaks, alu_peak, e0, e1, stream, dev):
    """4,000,000 x 512 BF16 rows, m = 32, L = 64: dense E2LSH on the tensor cores
    (GEMM 4M x 512 x 2048, BF16 family, and per-row-scaled FP8 rows with an E4M3
    family) with the exact boundary recheck, the BF16 family on the FP32 SIMT
    GEMM (bounded sample), and CS/HCS-E2LSH."""
    import torch
    from paper_2503_06737_gb300 import lsh, workloads
    wl = workloads.WORKLOADS["iid_4M_d512_bf16"]
    n, d, m, L = wl["n"], wl["d"], wl["m"], wl["L"]
    X = workloads.iid(n, d, seed=1238, device=dev, dtype=torch.bfloat16)
    keys = torch.empty((L, n), dtype=torch.int64, device=dev)
    mtx = lsh.dense_matrix(X)
    out = {"n": n, "d": d, "m": m, "L": L}

    def timed(fam, reps, mt=mtx, kk=keys):
        fam.hash_into(mt, None, lsh._ptr(kk), None)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fam.hash_into(mt, None, lsh._ptr(kk), None)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    flops = 2.0 * n * d * m * L
    ft = lsh.Family("e2lsh", d, m, L, w=wl["w"], seed=42, compute=lsh.BF16)
    tms = timed(ft, 5)
    log(f"tcgen05 dense: {tms:.3f} ms")
    st = ft.hash(X, keys=True, stats=True)["stats"]
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    out["dense_bf16_tcgen05"] = {"hash_ms": tms, "points_per_s": n / (tms / 1e3),
                                 "tflops": flops / (tms / 1e3) / 1e12,
                                 "tensor_frac": flops / (tms / 1e3) / 1e12 / bf16_peak,
                                 "flagged_per_entry": st["n_flagged"] / st["n_entries"],
                                 "mismatch_before_recheck": st["n_changed"] / st["n_entries"]}
    # per-row-scaled FP8 rows (scale = row amax / 448) with an E4M3 family on the tensor cores
    q8, sc8 = workloads.fp8_rows(X)
    f8 = lsh.Family("e2lsh", d, m, L, w=wl["w"], seed=42, compute=lsh.FP8_E4M3)
    m8 = lsh.dense_matrix(q8, sc8)
    fms = timed(f8, 5, m8)
    st8 = f8.hash(q8, keys=True, stats=True, row_scale=sc8)["stats"]
    out["dense_fp8_tcgen05"] = {"hash_ms": fms, "points_per_s": n / (fms / 1e3),
                                "tflops": flops / (fms / 1e3) / 1e12,
                                "tensor_frac_of_bf16_peak": flops / (fms / 1e3) / 1e12 / bf16_peak,
                                "flagged_per_entry": st8["n_flagged"] / st8["n_entries"],
                                "mismatch_before_recheck": st8["n_changed"] / st8["n_entries"],
                                "input": "E4M3 codes + FP32 row scale (2.05 GB)"}
    log(f"tcgen05 dense FP8: {fms:.3f} ms")
    f8.close()
    del q8, sc8, m8
    # the same BF16 family on the FP32 SIMT GEMM, on a 131,072-row sample (strided view forces that path)
    ns = 131072
    Xpad = torch.zeros((ns, d + 4), dtype=torch.bfloat16, device=dev)
    Xpad[:, :d] = X[:ns]
    ks = torch.empty((L, ns), dtype=torch.int64, device=dev)
    sms = timed(ft, 2, lsh.dense_matrix(Xpad[:, :d]), ks)
    out["dense_bf16_family_fp32_simt"] = {"hash_ms_per_1M_rows": sms * (1e6 / ns),
                                          "points_per_s": ns / (sms / 1e3),
                                          "tflops": 2.0 * ns * d * m * L / (sms / 1e3) / 1e12}
    ft.close()
    for kind, dims, mdims in (("cs_e2lsh", None, None), ("hcs_e2lsh", [16, 32], [4, 8])):
        fc = lsh.Family(kind, d, m, L, w=wl["w"], seed=42, dims=dims, mdims=mdims)
        cms = timed(fc, 3)
        out[kind] = {"hash_ms": cms, "points_per_s": n / (cms / 1e3),
                     "alu_frac": float(n) * d * L / (cms / 1e3) / 1e12 / alu_peak}
        fc.close()
    # recall@10 of 100 queries (database rows + N(0, 0.05^2) noise) against exact
    # k-NN, for the BF16 tensor-core family and the CS/HCS families (the FP8 path
    # hashes only: its rows are not kept for the rerank)
    from paper_2503_06737_gb300 import measure
    Qr, _ = workloads.noisy_queries(X, 100, 0.05, seed=9)
    truth, _ = measure.exact_knn(X, Qr, 10)
    truth = truth.cpu().numpy()
    for name, fargs in (("dense_bf16_tcgen05", dict(kind="e2lsh", compute=lsh.BF16)),
                        ("cs_e2lsh", dict(kind="cs_e2lsh")),
                        ("hcs_e2lsh", dict(kind="hcs_e2lsh", dims=[16, 32], mdims=[4, 8]))):
        fr = lsh.Family(d=d, m=m, L=L, w=wl["w"], seed=42, **fargs)
        ir = fr.build_index(X, keep_data=True)
        res = ir.query(Qr, k=10, stats=True)
        out[name]["recall10"] = measure.recall_at_k(res["ids"].cpu().numpy(), truth)
        out[name]["cand_per_query"] = res["stats"]["n_unique"] / 100.0
        ir.close()
        fr.close()
    del X, keys, Xpad, ks
    torch.cuda.empty_cache()
    return out


def m_sweep(X, e0, e1, stream):
    """The paper's space/time-versus-m comparison (Sec. 6, Table 1) on the
    1,000,000 x 960 mixture rows, L = 64: family bytes and hashing time (keys
    only) of CS-E2LSH, HCS-E2LSH (8x10x12) and the dense baseline on the
    tensor cores (BF16 copy of the rows and of G) as m grows."""
    import torch
    from paper_2503_06737_gb300 import lsh
    n, d, L = X.shape[0], X.shape[1], 64
    Xb = X.to(torch.bfloat16)
    keys = torch.empty((L, n), dtype=torch.int64, device=X.device)
    mtx, mtxb = lsh.dense_matrix(X), lsh.dense_matrix(Xb)
    hcs_m = {16: [2, 2, 4], 32: [2, 4, 4], 64: [4, 4, 4], 128: [4, 4, 8]}

    def timed(fam, mt, reps=5):
        fam.hash_into(mt, None, lsh._ptr(keys), None)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fam.hash_into(mt, None, lsh._ptr(keys), None)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"n": n, "d": d, "L": L, "rows": []}
    for m in (16, 32, 64, 128):
        row = {"m": m}
        f = lsh.Family("cs_e2lsh", d, m, L, w=4.0, seed=42)
        row["cs_ms"], row["cs_family_bytes"] = timed(f, mtx), L * d * 3
        f.close()
        f = lsh.Family("hcs_e2lsh", d, m, L, w=4.0, seed=42, dims=[8, 10, 12], mdims=hcs_m[m])
        row["hcs_ms"], row["hcs_family_bytes"] = timed(f, mtx), L * (8 + 10 + 12) * 3
        f.close()
        f = lsh.Family("e2lsh", d, m, L, w=4.0, seed=42, compute=lsh.BF16)
        row["dense_bf16_tcgen05_ms"], row["dense_family_bytes"] = timed(f, mtxb), d * m * L * 2
        f.close()
        out["rows"].append(row)
        log(f"m sweep m={m}: {row}")
    del Xb, keys
    torch.cuda.empty_cache()
    return out


def recall_protocol(dev, e0, e1, stream, reps=20, l_values=None, datasets=None):
    """The paper's indexing-quality protocol (Sec. 6) on synthetic stand-ins of
    its Gist (first 500,000 x 960) and Synthetic (50,000 x 10,000) datasets:
    the last 100 points are the queries, the rest the database; top-k = 50,
    m = 8; for L = 1, 2, ... until the average recall@50 reaches 0.99 (or
    L = 50) -- or the given L values -- each family kind is drawn reps times
    (seeds 42 + 1000 r), the index built and the 100 queries answered in one
    batch; average and spread of recall@50 and the total query time (CUDA
    events around the batch).  E2LSH kinds use w = 8 x the median distance of
    the 50th neighbour (the paper does not state w); SRP kinds are scored
    against the cosine top-50; HCS reshapes 960 = 8 x 10 x 12 (sketch
    2 x 2 x 2) and 10,000 = 100 x 100 (2 x 4)."""
    import numpy as np
    import torch
    from paper_2503_06737_gb300 import lsh, measure, workloads
    sets = datasets or ("gist_like_500k_d960", "synthetic_50k_d10000")
    out = {"k": 50, "m": 8, "queries": 100, "reps": reps, "datasets": {}}
    for name in sets:
        if name == "gist_like_500k_d960":
            X = workloads.gmm(500_000, 960, 64, seed=1239, device=dev)
            hcs = ([8, 10, 12], [2, 2, 2])
        else:
            X = workloads.iid(50_000, 10_000, seed=1240, device=dev)
            hcs = ([100, 100], [2, 4])
        D, Q = X[:-100].contiguous(), X[-100:].contiguous()
        truth, tdist = measure.exact_knn(D, Q, 50)
        truth = truth.cpu().numpy()
        # the paper does not state w: 8 x the median distance of the 50th
        # neighbour, where one E2LSH hash collides with probability ~0.9
        w = 8.0 * float(torch.median(tdist[:, -1]).item())
        # SRP kinds rank by cosine similarity: the same order as Euclidean on unit rows
        truth_cos, _ = measure.exact_knn(torch.nn.functional.normalize(D.float(), dim=1),
                                         torch.nn.functional.normalize(Q.float(), dim=1), 50)
        truth_cos = truth_cos.cpu().numpy()
        rows = []
        for kind in ("e2lsh", "cs_e2lsh", "hcs_e2lsh", "srp", "cs_srp", "hcs_srp"):
            hc = kind.startswith("hcs")
            for Lt in (l_values or range(1, 51)):
                recs, qms, cand = [], [], 0.0
                for r in range(reps):
                    fam = lsh.Family(kind, D.shape[1], 8, Lt, w=w, seed=42 + 1000 * r, dims=hcs[0] if hc else None,
                                     mdims=hcs[1] if hc else None)
                    idx = fam.build_index(D, keep_data=True)
                    idx.query(Q, k=50)  # first call: temporaries from the pool
                    torch.cuda.synchronize()
                    e0.record(stream)
                    res = idx.query(Q, k=50)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    qms.append(e0.elapsed_time(e1))
                    recs.append(measure.recall_at_k(res["ids"].cpu().numpy(), truth_cos if "srp" in kind else truth))
                    if r == 0:
                        cand = idx.query(Q, k=50, stats=True)["stats"]["n_unique"] / 100.0
                    idx.close()
                    fam.close()
                rows.append({"kind": kind, "L": Lt, "recall50": float(np.mean(recs)),
                             "recall50_std": float(np.std(recs)), "query_ms": float(np.mean(qms)),
                             "cand_per_query": cand})
                if l_values is None and np.mean(recs) >= 0.99:
                    break
        out["datasets"][name] = {"n_database": int(D.shape[0]), "d": int(D.shape[1]), "w": w, "rows": rows}
        log(f"recall protocol {name} done")
        del X, D, Q
        torch.cuda.empty_cache()
    return out


def serving_bench(dev, e0, e1, stream, max_requests=200, max_cand=5e6, seconds_per_load=8.0):
    """Serving workload: 10,000,000 x 128 FP16 points from a 1,024-component
    mixture resident on the GPU; HCS-E2LSH (8 x 16 -> 4 x 4, m = 16) and
    CS-E2LSH (m = 12), L = 32, each with w the smallest value on a grid that
    reaches recall@10 >= 0.9 against exact k-NN on 200 noisy queries; Poisson
    arrivals of log-uniform 1..4096-query batches at 25/50/90% of the measured
    saturation throughput through the continuous-batching loop."""
    import numpy as np
    import torch
    from paper_2503_06737_gb300 import lsh, measure, workloads
    wl = workloads.WORKLOADS["gmm1024_10M_d128_f16"]
    X = workloads.gmm(wl["n"], wl["d"], wl["components"], seed=1237, device=dev, dtype=torch.float16)
    Qpool, _ = workloads.noisy_queries(X, 20000, wl["query_sigma"], seed=7)
    Qt = Qpool[:200].contiguous()
    truth, _ = measure.exact_knn(X, Qt, 10)
    truth = truth.cpu().numpy()
    rng = np.random.default_rng(11)
    out = {"n": wl["n"], "d": wl["d"], "L": wl["L"], "queries": "database rows + N(0, 0.05^2) noise",
           "batch_sizes": "floor(exp(U[0, ln 4097)))"}
    # context: exact k-NN by brute force on the same GPU (FP32 products over the
    # whole database, FP64 refinement of the best) for one 4096-query batch
    Qb = Qpool[:4096].contiguous()
    measure.exact_knn(X, Qb[:64], 10)
    torch.cuda.synchronize()
    e0.record(stream)
    measure.exact_knn(X, Qb, 10)
    e1.record(stream)
    torch.cuda.synchronize()
    bms = e0.elapsed_time(e1)
    out["exact_knn_bruteforce"] = {"batch": 4096, "batch_ms": bms, "qps": 4096 / (bms / 1e3), "recall10": 1.0,
                                   "note": "torch FP32 matrix products + top-k over all 10,000,000 rows"}
    log(f"serving: brute-force exact k-NN {4096 / (bms / 1e3):.0f} queries/s")
    # the same scan with TF32 tensor-core products (the FP64 refinement of each
    # chunk's best 2k keeps the order exact unless TF32 moves a neighbour out)
    tf32_prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        e0.record(stream)
        ids_tf, _ = measure.exact_knn(X, Qb, 10)
        e1.record(stream)
        torch.cuda.synchronize()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32_prev
    tms = e0.elapsed_time(e1)
    ids_fp, _ = measure.exact_knn(X, Qb[:256], 10)
    out["exact_knn_bruteforce_tf32"] = {
        "batch": 4096, "batch_ms": tms, "qps": 4096 / (tms / 1e3),
        "recall10_vs_fp32": measure.recall_at_k(ids_tf[:256].cpu().numpy(), ids_fp.cpu().numpy()),
        "note": "TF32 tensor-core products + torch top-k (which takes most of the time) + FP64 refinement"}
    log(f"serving: brute-force k-NN with TF32 products {4096 / (tms / 1e3):.0f} queries/s")
    for kind, m, dims, mdims in (("hcs_e2lsh", wl["m_hcs"], wl["hcs_dims"], wl["hcs_mdims"]),
                                 ("cs_e2lsh", wl["m_cs"], None, None)):
        chosen = None
        tried = []
        best = None
        for w in (4.0, 8.0, 16.0, 24.0, 32.0, 36.0, 40.0, 42.0, 44.0, 46.0, 48.0, 56.0, 64.0, 96.0):
            fam = lsh.Family(kind, wl["d"], m, wl["L"], w=w, seed=42, dims=dims, mdims=mdims)
            idx = fam.build_index(X, keep_data=True)
            res = idx.query(Qt, k=10, stats=True)
            rec = measure.recall_at_k(res["ids"].cpu().numpy(), truth)
            cpq = res["stats"]["n_unique"] / 200.0
            tried.append({"w": w, "recall10": rec, "cand_per_query": cpq})
            log(f"serving {kind} w={w}: recall@10 {rec:.3f}, {cpq:.0f} candidates/query")
            if rec >= 0.9 or cpq > max_cand:
                chosen = (w, fam, idx, rec, res["stats"])
                break
            idx.close()
            fam.close()
        entry = {"w_grid": tried}
        if chosen is None:
            out[kind] = entry
            continue
        w, fam, idx, rec, qst = chosen
        mtx = lsh.dense_matrix(X)
        e0.record(stream)
        idx.rebuild_into(mtx)
        e1.record(stream)
        torch.cuda.synchronize()
        entry.update({"w": w, "recall10": rec, "m": m, "cand_per_query": qst["n_unique"] / 200.0,
                      "build_ms": e0.elapsed_time(e1),
                      "recall_target_met": rec >= 0.9})
        srv = lsh.Server(idx, max_batch=4096, slots=4, k=10, use_graphs=True)
        measure.run_load(srv, Qpool, measure.log_uniform_sizes(40, 4096, rng), None, rng,
                         max_seconds=seconds_per_load)  # capture graphs
        sat, lat = measure.run_load(srv, Qpool, measure.log_uniform_sizes(max_requests, 4096, rng), None, rng,
                                    max_seconds=seconds_per_load)
        entry["saturation_qps"] = sat
        log(f"serving {kind}: saturation {sat:.0f} queries/s")
        loads = []
        for frac in (0.25, 0.5, 0.9):
            srv.stats(reset=True)
            qps, lat = measure.run_load(srv, Qpool, measure.log_uniform_sizes(max_requests, 4096, rng),
                                        frac * sat, rng, max_seconds=seconds_per_load)
            log(f"serving {kind}: load {frac:.2f} -> {qps:.0f} q/s, p50 {np.percentile(lat, 50):.2f} ms, "
                f"p99 {np.percentile(lat, 99):.2f} ms")
            loads.append({"offered_qps": frac * sat, "achieved_qps": qps, "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99)), "requests": int(len(lat)),
                          "admitted_peak": srv.stats()["admitted_peak"]})
        entry["loads"] = loads
        srv.close()
        idx.close()
        fam.close()
        out[kind] = entry
    del X, Qpool
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gmm64_1M_d960")
    ap.add_argument("--kind", default="cs_e2lsh")
    ap.add_argument("--no-extras", action="store_true", help="skip the per-family hashing lines")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving workload")
    ap.add_argument("--recall-protocol", action="store_true",
                    help="run the paper's full recall protocol (20 repetitions, L up to 50) in the extras")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2503_06737_gb300 import build as libbuild
    libbuild.build()
    from paper_2503_06737_gb300 import lsh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    peaks, peak_src = _peaks()
    wl, fam_args = _workload(args.workload, args.kind)
    n, d, L, m = wl["n"], wl["d"], fam_args["L"], fam_args["m"]
    X = _make_X(wl, seed=shard_seed(rank), device=dev)
    x_gb = X.numel() * X.element_size() / 1e9
    fam = lsh.Family(**fam_args)
    idx = fam.build_index(X, keep_data=False)
    mtx = lsh.dense_matrix(X)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    log("data ready, warm-up")
    for _ in range(args.warmup):
        idx.rebuild_into(mtx)
    barrier()
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    sel = f"GPU-{uuid}" if uuid is not None else os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]
    clocks = ClockSampler(sel)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = lsh.launch_count()
    t_wall0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        idx.rebuild_into(mtx)
    e1.record(stream)
    barrier()
    t_wall1 = time.time()
    launches = lsh.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    value = job_throughput(world, n, ms)
    log(f"timed region: {ms:.3f} ms/step")

    # ---- dominant kernel alone: the hashing launch (keys only) ----
    keys = torch.empty((L, n), dtype=torch.int64, device=dev)
    for _ in range(3):
        fam.hash_into(mtx, None, lsh._ptr(keys), None)
    barrier()
    kst = max(10, args.steps // 2)
    e0.record(stream)
    for _ in range(kst):
        fam.hash_into(mtx, None, lsh._ptr(keys), None)
    e1.record(stream)
    torch.cuda.synchronize()
    hash_ms = e0.elapsed_time(e1) / kst
    adds = float(n) * d * L                     # signed adds: one per (coordinate, table)
    bytes_alg = float(n) * d * X.element_size() + float(n) * L * 8
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = props.multi_processor_count
    alu_peak = nsm * 128 * sm_max * 1e6 / 1e12  # FP32 adds/s in T/s
    achieved = adds / (hash_ms / 1e3) / 1e12
    traffic = _profiled_traffic("sketch_dense_kernel", args.workload)
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": traffic,
                "kernel": "sketch_dense_kernel (CS/HCS hash, all tables, keys only)",
                "plan": fam.sketch_plan(n, X.dtype),
                "kernel_ms": hash_ms, "peak_source": f"{nsm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz",
                "hbm_view": {"algorithmic_bytes": bytes_alg,
                             "achieved_gbs": bytes_alg / (hash_ms / 1e3) / 1e9,
                             "peak_gbs": peaks["hbm_gbs"],
                             "frac": bytes_alg / (hash_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                             "peak_source": peak_src},
                # one 4-byte x operand from shared memory per (coordinate, table):
                # 128 B/clk/SM of shared-memory return = 32 operands per clock per SM
                "smem_operand_view": {"achieved_per_s": adds / (hash_ms / 1e3),
                                      "peak_per_s": nsm * 32 * sm_max * 1e6,
                                      "frac": adds / (hash_ms / 1e3) / (nsm * 32 * sm_max * 1e6),
                                      "peak_source": f"{nsm} SMs x 32 x 4-byte operands/clk x {sm_max:.0f} MHz"}}
    t_wall2 = time.time()

    # ---- end to end through the public API with host buffers ----
    Xh, host_buffer = _pinned_near_gpu(X.shape, X.dtype, dev)
    Xh.copy_(X)
    nb_host = torch.empty(L, dtype=torch.int64, pin_memory=True)
    import ctypes
    e2e_steps = max(5, args.steps // 5)

    def e2e_step():
        # lsh_index_rebuild_host: the rows stream from pinned host memory in
        # chunks whose copies overlap the hashing of the previous chunk
        idx.rebuild_from_host(Xh)
        # the step's result: bucket counts of every table
        lsh._check(lsh.lib().lsh_index_info(idx.handle, None, ctypes.c_void_p(nb_host.data_ptr())))

    for _ in range(2):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e = {"value": job_throughput(world, n, e2e_ms), "unit": "points/s",
           "h2d_bytes_per_step": int(X.numel() * X.element_size()), "d2h_bytes_per_step": int(L * 8),
           "ms_per_step": e2e_ms, "host_buffer": host_buffer}
    del Xh

    # ---- per-family hashing throughput (keys only), same workload ----
    variants = {}
    if not args.no_extras:
        for kind in ("cs_e2lsh", "hcs_e2lsh", "cs_srp", "hcs_srp"):
            _, fa = _workload(args.workload, kind)
            f2 = lsh.Family(**fa)
            for _ in range(3):
                f2.hash_into(mtx, None, lsh._ptr(keys), None)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(10):
                f2.hash_into(mtx, None, lsh._ptr(keys), None)
            e1.record(stream)
            torch.cuda.synchronize()
            kms = e0.elapsed_time(e1) / 10
            st = f2.hash(X, keys=True, stats=True)["stats"]
            variants[kind] = {"hash_ms": kms, "points_per_s": n / (kms / 1e3),
                              "alu_frac": adds / (kms / 1e3) / 1e12 / alu_peak,
                              "hbm_frac": bytes_alg / (kms / 1e3) / 1e9 / peaks["hbm_gbs"],
                              "flagged_per_entry": st["n_flagged"] / max(1, st["n_entries"]),
                              "changed": st["n_changed"]}
            f2.close()
        # the same hash with the int32 codes [n, L, m] written too (12.8 GB at the
        # headline): the HBM view of hashcode generation
        codes = torch.empty((n, L, m), dtype=torch.int32, device=dev)
        fam.hash_into(mtx, lsh._ptr(codes), lsh._ptr(keys), None)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            fam.hash_into(mtx, lsh._ptr(codes), lsh._ptr(keys), None)
        e1.record(stream)
        torch.cuda.synchronize()
        cms = e0.elapsed_time(e1) / 3
        cbytes = bytes_alg + float(codes.numel()) * 4
        variants["cs_e2lsh_codes_out"] = {"hash_ms": cms, "points_per_s": n / (cms / 1e3),
                                          "algorithmic_bytes": cbytes,
                                          "hbm_frac": cbytes / (cms / 1e3) / 1e9 / peaks["hbm_gbs"],
                                          "note": "keys and int32 codes [n, L, m] written"}
        del codes
        torch.cuda.empty_cache()
        # CSSRP-L (Table 1): l bins per coordinate, l times the count sketch's adds
        for lc in (2, 4):
            fa = dict(_workload(args.workload, "cs_srp")[1], kind="csl_srp", l=lc)
            f2 = lsh.Family(**fa)
            for _ in range(3):
                f2.hash_into(mtx, None, lsh._ptr(keys), None)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(10):
                f2.hash_into(mtx, None, lsh._ptr(keys), None)
            e1.record(stream)
            torch.cuda.synchronize()
            kms = e0.elapsed_time(e1) / 10
            variants[f"csl_srp_l{lc}"] = {"hash_ms": kms, "points_per_s": n / (kms / 1e3),
                                          "alu_frac": lc * adds / (kms / 1e3) / 1e12 / alu_peak,
                                          "note": f"CSSRP-L, {lc} nonzeros per column of the sketch matrix"}
            f2.close()
        log("per-family hashing done")
        variants["uneven_batches_gmm64_d960"] = uneven_batches(X, keys, e0, e1, stream)
        log("uneven batches done")
        variants.update(extra_variants(args, X, keys, peaks, alu_peak, e0, e1, stream))
        log("extra variants done")
        del keys
        torch.cuda.empty_cache()
        variants["m_sweep_gmm64_1M_d960"] = m_sweep(X, e0, e1, stream)
        keys = None
        # the paper's recall protocol: the full one (20 repetitions, L = 1, 2, ...
        # until recall 0.99) with --recall-protocol, else two repetitions at five L
        variants["recall_protocol"] = (recall_protocol(dev, e0, e1, stream) if args.recall_protocol else
                                       recall_protocol(dev, e0, e1, stream, reps=2, l_values=(1, 5, 10, 20, 50)))
    if not args.no_serving and world == 1:
        idx.close()
        fam.close()
        del X, keys, mtx
        torch.cuda.empty_cache()
        variants["serving_gmm1024_10M_d128_f16"] = serving_bench(dev, e0, e1, stream)
    clocks.stop()
    clk = clocks.summary(t_wall0, t_wall2)

    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        rate, rows, t, cores = oracle_sample_rate(wl, fam_args, target_s=args.cpu_seconds)
        cpu = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
               "sample": f"{rows} rows of {args.workload}: {fam_args['kind']} hash + index, FP64, {t:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "kind": fam_args["kind"], "n_per_gpu": n, "d": d,
                       "m": m, "L": L, "w": fam_args["w"],
                       "step": "lsh_index_rebuild: hash (FP32 + FP64 recheck) + bucket sort + segmentation",
                       "l2": "inputs larger than L2 (%.2f GB per GPU)" % x_gb},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "variants": variants,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
