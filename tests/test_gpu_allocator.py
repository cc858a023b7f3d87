"""Device memory of a context comes from the caller's allocator: with the
binding's default (torch's caching allocator) every byte the library owns is
visible to torch, and goes back to it on close; with allocator=None the
library allocates for itself and torch sees nothing."""
import numpy as np
import pytest
import torch

from oracle import tucker_oracle as O
from paper_1804_09494_gb300.tucker import Tucker
from tests.gpu_cases import case, factors

pytestmark = pytest.mark.gpu


def _inputs():
    c = case((3000, 2000, 500), 200_000, (1.1, 1.1, 1.1), "lognormal", seed=43)
    idx = torch.from_numpy(c["idx"]).cuda()
    vals = torch.from_numpy(c["vals"]).cuda()
    return c, idx, vals


def test_context_memory_comes_from_torch_and_goes_back():
    c, idx, vals = _inputs()
    K = (10, 10, 10)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    tk = Tucker(idx, vals, c["L"], K, prec="fp32")
    torch.cuda.synchronize()
    owned = tk.memory()
    assert owned > 0
    assert torch.cuda.memory_allocated() - base >= owned
    # the context works on that memory: one invocation against the oracle
    Fd, Fo = factors(c["L"], K, 3, "fp32")
    F = [f.clone() for f in Fd]
    G, fit = tk.hooi_iter(F)
    Fr = O.hooi_invocation(c["L"], c["idx"], c["vals"].astype(np.float64), Fo)
    fo = O.fit(c["vals"].astype(np.float64), O.core(c["L"], c["idx"], c["vals"].astype(np.float64), Fr))
    assert abs(fit - fo) <= 1e-6
    # the adjoint's workspace also comes from torch, on its first call
    before = torch.cuda.memory_allocated()
    W = torch.randn(tk.R[0], tk.khat(0), device="cuda")
    tk.ttm_chain_backward(0, Fd, W)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() > before
    assert torch.cuda.memory_allocated() - base >= tk.memory()
    tk.close()
    torch.cuda.synchronize()
    del W, G, F
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() <= base + 4 * 1024 * 1024  # only the test's own small tensors remain


def test_library_allocator_leaves_torch_untouched():
    c, idx, vals = _inputs()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    tk = Tucker(idx, vals, c["L"], (10, 10, 10), prec="fp32", allocator=None)
    torch.cuda.synchronize()
    assert tk.memory() > 0
    assert torch.cuda.memory_allocated() == base
    tk.close()
