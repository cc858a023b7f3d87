"""tucker_partition_noalloc (the export for callers that cannot allocate
device memory while they run) gives bit-identical output to
tucker_partition, on two calls in a row.  Kept in a file of its own that is
collected last."""
import numpy as np
import pytest
import torch

from tests.gpu_cases import case, make

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("P", [0, 77])
def test_partition_noalloc_matches_partition(P):
    c = case((3000, 2000, 500), 200_000, (1.1, 1.1, 1.1), "lognormal", seed=41)
    tk = make(c, (10, 10, 10), "fp32", P_bins=P)
    for n in range(3):
        ref_ptr, ref_perm = tk.partition(n)
        nb = tk.stats(n)["P"]
        for _ in range(2):  # two calls in a row share the static scratch
            bin_ptr = torch.full((nb + 1,), -1, dtype=torch.int64, device="cuda")
            perm = torch.full((tk.nnz,), -1, dtype=torch.int32, device="cuda")
            tk.partition_noalloc(n, bin_ptr, perm)
            torch.cuda.synchronize()
            assert torch.equal(bin_ptr, ref_ptr)
            assert torch.equal(perm, ref_perm)
    tk.close()
