"""Measurement support for the serving benchmark: exact k-NN ground truth for
recall@k, bin-width tuning, and a Poisson load generator driving the serving
loop.  None of this is on the hashing / indexing / query path; the ground
truth uses torch matrix products on the GPU (a ground-truth generator only,
checked against the FP64 oracle's brute force in tests/test_gpu_measure.py).
"""
from __future__ import annotations

import math
import threading
import time

import numpy as np
import torch


def exact_knn(X: torch.Tensor, Q: torch.Tensor, k: int, chunk: int = 1 << 20):
    """Exact Euclidean k-NN ids [q, k] (ties by id) of Q among the rows of X,
    from FP32 ||x||^2 - 2 q.x + ||q||^2 over row chunks, refined in FP64 on the
    2k best of every chunk so the returned order is exact in FP64."""
    q = Q.shape[0]
    Qf = Q.to(torch.float32)
    best_d = torch.full((q, 0), float("inf"), device=X.device, dtype=torch.float64)
    best_i = torch.zeros((q, 0), device=X.device, dtype=torch.int64)
    qq = (Qf * Qf).sum(1, keepdim=True)
    for s in range(0, X.shape[0], chunk):
        Xc = X[s:s + chunk].to(torch.float32)
        d2 = (Xc * Xc).sum(1)[None, :] - 2.0 * (Qf @ Xc.T) + qq
        kk = min(2 * k, Xc.shape[0])
        _, ci = torch.topk(d2, kk, dim=1, largest=False)
        cand = Xc[ci].to(torch.float64)                       # [q, kk, d]
        dd = ((cand - Q.to(torch.float64)[:, None, :]) ** 2).sum(-1)
        best_d = torch.cat([best_d, dd], 1)
        best_i = torch.cat([best_i, ci + s], 1)
        # keep the k best by (distance, id)
        order = torch.argsort(best_i, dim=1, stable=True)
        best_d = torch.gather(best_d, 1, order)
        best_i = torch.gather(best_i, 1, order)
        order = torch.argsort(best_d, dim=1, stable=True)[:, :k]
        best_d = torch.gather(best_d, 1, order)
        best_i = torch.gather(best_i, 1, order)
    return best_i, best_d.sqrt()


def recall_at_k(found: np.ndarray, truth: np.ndarray) -> float:
    """Mean over queries of |S n S'| / |S| (Sec. 6), S the exact top-k."""
    r = []
    for f, t in zip(found, truth):
        s = set(t.tolist())
        r.append(len(s & set(x for x in f.tolist() if x >= 0)) / len(s))
    return float(np.mean(r))


def log_uniform_sizes(n: int, hi: int, rng: np.random.Generator):
    """Batch sizes floor(exp(U[0, ln(hi + 1)))), i.e. log-uniform on 1..hi."""
    return np.clip(np.floor(np.exp(rng.uniform(0, math.log(hi + 1), size=n))).astype(np.int64), 1, hi)


def run_load(server, Qpool: torch.Tensor, sizes, rate_qps: float | None, rng: np.random.Generator,
             max_seconds: float | None = None):
    """Submit batches of the given sizes (rows drawn from Qpool) with Poisson
    arrivals at `rate_qps` queries per second (None: back to back, keeping the
    loop saturated); a second thread waits for completions.  Returns
    (queries/s over the run, per-request latencies in ms).  With max_seconds,
    no request is submitted after that much time has passed."""
    Qh = Qpool.cpu().contiguous()
    nq = Qh.shape[0]
    starts = rng.integers(0, max(1, nq - int(max(sizes))), size=len(sizes))
    tickets = []
    lock = threading.Lock()
    done_evt = threading.Event()
    lat = []

    def waiter():
        i = 0
        while True:
            with lock:
                have = i < len(tickets)
                t = tickets[i] if have else None
                finished = done_evt.is_set() and i >= len(tickets)
            if have:
                _, _, ms = server.wait(t)
                lat.append(ms)
                i += 1
            elif finished:
                break
            else:
                time.sleep(5e-5)

    th = threading.Thread(target=waiter)
    th.start()
    t0 = time.perf_counter()
    next_t = t0
    total = 0
    for b, s0 in zip(sizes, starts):
        if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
            break
        if rate_qps:
            next_t += rng.exponential(b / rate_qps)
            dt = next_t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        tk = server.submit(Qh[s0:s0 + b])
        with lock:
            tickets.append(tk)
        total += int(b)
    done_evt.set()
    th.join()
    el = time.perf_counter() - t0
    return total / el, np.array(lat) if lat else np.zeros(1)
