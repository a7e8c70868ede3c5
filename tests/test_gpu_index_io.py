"""lsh_index_save / lsh_index_load through the C ABI: the loaded tables equal
the saved ones array for array, queries on the loaded index return the same
results, and a family other than the file's, or a missing file, is refused."""
import numpy as np
import pytest
import torch

from paper_2503_06737_gb300 import lsh, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,dims,mdims,dtype,l", [("cs_e2lsh", None, None, torch.float32, 1),
                                                     ("hcs_srp", [8, 8], [4, 4], torch.float16, 1),
                                                     ("csl_srp", None, None, torch.float32, 3)])
def test_save_load_roundtrip(tmp_path, kind, dims, mdims, dtype, l):
    X = workloads.gmm(5000, 64, 8, seed=21, device="cpu", dtype=dtype).cuda()
    fam = lsh.Family(kind, 64, 16, 6, w=4.0, seed=5, dims=dims, mdims=mdims, l=l)
    idx = fam.build_index(X, keep_data=True)
    path = tmp_path / "index.bin"
    idx.save(path)
    fam2 = lsh.Family(kind, 64, 16, 6, w=4.0, seed=5, dims=dims, mdims=mdims, l=l)
    loaded = lsh.load_index(fam2, path)
    a, b = idx.export(), loaded.export()
    for key in ("ids", "nb", "offsets"):
        assert np.array_equal(a[key], b[key]), key
    for t in range(6):
        nb = int(a["nb"][t])
        assert np.array_equal(a["ukeys"][t, :nb], b["ukeys"][t, :nb])
    Q = X[::97].contiguous()
    r1, r2 = idx.query(Q, k=10), loaded.query(Q, k=10)
    torch.cuda.synchronize()
    assert torch.equal(r1["ids"], r2["ids"]) and torch.equal(r1["dist"], r2["dist"])
    other = lsh.Family(kind, 64, 16, 6, w=4.0, seed=6, dims=dims, mdims=mdims)
    with pytest.raises(lsh.LshError) as e:
        lsh.load_index(other, path)
    assert e.value.status == 1  # LSH_EINVAL: another family
    if kind == "csl_srp":
        with pytest.raises(lsh.LshError) as e:
            lsh.load_index(lsh.Family(kind, 64, 16, 6, w=4.0, seed=5, l=2), path)
        assert e.value.status == 1  # another number of nonzeros per column
    with pytest.raises(lsh.LshError) as e:
        lsh.load_index(fam2, tmp_path / "missing.bin")
    assert e.value.status == 8  # LSH_EIO
    loaded.close()
    idx.close()
