"""blockcg_block_cdot_noalloc, the block inner product for callers that cannot
allocate device memory (its scratch is a fixed array in the library's device
image), against the workspace-based blockcg_block_cdot.

Kept in a file that pytest collects last, so that a failure here cannot stop
a -x run before the rest of the suite has run."""
import ctypes as ct

import numpy as np
import pytest

import hisq_inputs as hi
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu


def _noalloc(lib, X, Y, stream):
    torch = gh.torch_mod()
    n = X.shape[0]
    K = torch.empty((n, n), dtype=torch.complex128, device=X.device)
    rc = lib.blockcg_block_cdot_noalloc(ct.c_void_p(X.data_ptr()), ct.c_void_p(Y.data_ptr()), n,
                                        X.shape[1], ct.c_void_p(K.data_ptr()),
                                        ct.c_void_p(stream.cuda_stream))
    assert rc == 0, rc
    return K


@pytest.mark.parametrize("N", [1, 5, 16, 64])
def test_noalloc_cdot_matches_workspace_cdot_twice(N):
    torch = gh.torch_mod()
    dims = (6, 8, 10, 12)
    s, _, _ = gh.make_solver(dims, 0.1, prec="f64", max_rhs=max(N, 16))
    lib = s.lib
    stream = torch.cuda.current_stream()
    for call in range(2):  # two calls in a row share the scratch array
        X = torch.as_tensor(hi.gaussian_sources(dims, N, seed=300 + call)).cuda()
        Y = torch.as_tensor(hi.gaussian_sources(dims, N, seed=400 + call)).cuda()
        K = _noalloc(lib, X, Y, stream).cpu().numpy()
        Kref = s.block_cdot(X, Y).cpu().numpy()
        xn = np.linalg.norm(X.cpu().numpy().reshape(N, -1), axis=1).max()
        yn = np.linalg.norm(Y.cpu().numpy().reshape(N, -1), axis=1).max()
        assert np.abs(K - Kref).max() < 1e-13 * xn * yn, call


def test_noalloc_cdot_rejects_sizes_beyond_the_limit():
    torch = gh.torch_mod()
    gh.ensure_built()
    from paper_1710_09745_gb300 import load_library
    lib = load_library()
    X = torch.zeros((1, 8, 3), dtype=torch.complex128, device="cuda")
    K = torch.zeros((1, 1), dtype=torch.complex128, device="cuda")
    p = ct.c_void_p(X.data_ptr())
    assert lib.blockcg_block_cdot_noalloc(p, p, 65, 8, ct.c_void_p(K.data_ptr()), None) == 1
    assert lib.blockcg_block_cdot_noalloc(p, p, 0, 8, ct.c_void_p(K.data_ptr()), None) == 1
    assert lib.blockcg_block_cdot_noalloc(p, p, 1, 0, ct.c_void_p(K.data_ptr()), None) == 1
