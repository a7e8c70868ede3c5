"""The serving benchmark's ground truth (measure.exact_knn) against the FP64
oracle's brute-force k-NN on a subset, and the recall definition of Sec. 6."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_06737_gb300 import measure, workloads

from gpu_helpers import to_oracle

pytestmark = pytest.mark.gpu


def test_exact_knn_matches_oracle_bruteforce():
    X = workloads.gmm(30000, 128, 64, seed=3, device="cpu", dtype=torch.float16).cuda()
    Q, _ = workloads.noisy_queries(X, 25, 0.05, seed=4)
    ids, dist = measure.exact_knn(X, Q, 10, chunk=7000)
    Xh, dt = to_oracle(X)
    Qh, dq = to_oracle(Q)
    oids, odist = oracle.bruteforce_knn(Xh, Qh, 10, 0, dtype=dt, dtype_q=dq)
    assert np.array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_allclose(dist.cpu().numpy(), odist, rtol=1e-12)


def test_recall_definition():
    truth = np.array([[1, 2, 3, 4], [5, 6, 7, 8]])
    found = np.array([[1, 2, 9, -1], [8, 7, 6, 5]])
    assert measure.recall_at_k(found, truth) == pytest.approx((2 / 4 + 1.0) / 2)
