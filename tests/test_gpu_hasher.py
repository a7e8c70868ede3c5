"""lsh_hasher: replayed hashing of uneven batches through captured CUDA graphs.
Every batch's keys must equal lsh_hash's bit for bit (and the oracle's on a
sampled batch), batches of one size bucket must share one captured graph,
and out-of-contract calls must be refused before any device work."""
import numpy as np
import pytest
import torch

from paper_2503_06737_gb300 import lsh, workloads

from gpu_helpers import oracle_keys

pytestmark = pytest.mark.gpu


def _rows(n, d, seed, dtype):
    return workloads.gmm(n, d, 16, seed=seed, device="cpu", dtype=dtype).cuda()


@pytest.mark.parametrize("kind,d,m,L,dims,mdims,dtype", [
    ("cs_e2lsh", 960, 64, 13, None, None, torch.float32),
    ("hcs_srp", 200, 16, 9, [10, 20], [4, 4], torch.bfloat16),
    ("cs_srp", 128, 96, 5, None, None, torch.float16),
    ("hcs_e2lsh", 128, 16, 32, [8, 16], [4, 4], torch.float16),
])
def test_hasher_uneven_batches_equal_lsh_hash(kind, d, m, L, dims, mdims, dtype):
    fam = lsh.Family(kind, d, m, L, w=4.0, seed=77, dims=dims, mdims=mdims)
    h = lsh.Hasher(fam, dtype=dtype, max_rows=140000)
    # sizes: one bucket twice (9,000 and 12,000 -> 16,384), the smallest
    # bucket (1, 100, 8,191), and two larger buckets (131,077 and 70,000 rows)
    sizes = [9000, 12000, 1, 100, 8191, 131077, 70000, 16384]
    big = _rows(max(sizes) + len(sizes), d, seed=d + L, dtype=dtype)
    for i, n in enumerate(sizes):
        X = big[i:i + n]  # different pointers, same stride
        assert X.shape[0] == n
        got = h.run(X)
        want = fam.hash(X, keys=True)["keys"]
        torch.cuda.synchronize()
        assert torch.equal(got, want), (kind, n)
    info = h.info()
    assert info["replays"] == len(sizes)
    # buckets (log2 rows): 14, 13 (x3), 18, 17, 14 -- 9,000 / 12,000 / 16,384 share one
    assert info["captures"] == 4, info
    h.close()
    fam.close()


def test_hasher_keys_against_oracle_and_strided_keys():
    fa = dict(kind="cs_e2lsh", d=300, m=32, L=7, w=2.0, seed=5)
    fam = lsh.Family(fa["kind"], fa["d"], fa["m"], fa["L"], w=fa["w"], seed=fa["seed"])
    X = workloads.gmm(9001, 300, 8, seed=3, device="cpu")
    h = lsh.Hasher(fam, dtype=torch.float32, max_rows=20000)
    keys = torch.full((7, 9100), -1, dtype=torch.int64, device="cuda")  # key_ld > n
    h.run(X.cuda(), keys=keys)
    torch.cuda.synchronize()
    got = keys[:, :9001].cpu().numpy().view(np.uint64)
    assert np.array_equal(got, oracle_keys(fa, X))
    assert (keys[:, 9001:] == -1).all()  # nothing written past n
    h.close()
    fam.close()


def test_hasher_refusals():
    fam = lsh.Family("cs_srp", 64, 8, 4, seed=1)
    h = lsh.Hasher(fam, dtype=torch.float32, max_rows=1000)
    X = torch.zeros((1001, 64), device="cuda")
    with pytest.raises(lsh.LshError) as e:
        h.run(X)  # more rows than max_rows
    assert e.value.status == 1
    with pytest.raises(lsh.LshError) as e:
        h.run(X.view(torch.uint8).view(-1)[4:4 + 10 * 256].view(torch.float32).view(10, 64))  # misaligned
    assert e.value.status == 1
    assert h.info() == dict(captures=0, replays=0)
    h.close()
    dense = lsh.Family("e2lsh", 64, 8, 4, seed=1)
    with pytest.raises(lsh.LshError) as e:
        lsh.Hasher(dense, dtype=torch.float32)
    assert e.value.status == 6  # LSH_EUNSUPPORTED
    fam.close()
    dense.close()
