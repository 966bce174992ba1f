"""blockcg_block_cdot_noalloc, the block inner product for callers that cannot
allocate device memory (its scratch is a fixed array in the library's device
image), against the oracle's block_cdot (plain NumPy FP64) and against the
workspace-based blockcg_block_cdot.

Kept in a file that pytest collects last, so that a failure here cannot stop
a -x run before the rest of the suite has run."""
import ctypes as ct

import numpy as np
import pytest

import hisq_inputs as hi
from oracle import block as oblock
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


# N = 17 and 40: more Gram entries than threads of a CTA, so threads hold a
# ragged number of entries (1 or 2)
@pytest.mark.parametrize("N", [1, 5, 16, 17, 40, 64])
def test_noalloc_cdot_matches_oracle_twice(N):
    """Two calls in a row (they share the scratch array), each compared
    element by element with the oracle's K = X^dag Y and with the
    workspace-based entry point.  Tolerance: native FP64 sums of
    3 Vh products, rounding bound ~ 3 Vh u |x_i| |y_j| with u = 2^-53."""
    torch = gh.torch_mod()
    dims = (6, 8, 10, 12)
    vh = int(np.prod(dims)) // 2
    s, _, _ = gh.make_solver(dims, 0.1, prec="f64_native", max_rhs=max(N, 16))
    lib = s.lib
    stream = torch.cuda.current_stream()
    for call in range(2):
        Xn = hi.gaussian_sources(dims, N, seed=300 + call)
        Yn = hi.gaussian_sources(dims, N, seed=400 + call)
        X = torch.as_tensor(Xn).cuda()
        Y = torch.as_tensor(Yn).cuda()
        K = _noalloc(lib, X, Y, stream).cpu().numpy()
        Kref = oblock.block_cdot(oblock.as_columns(Xn), oblock.as_columns(Yn))
        xn = np.linalg.norm(Xn.reshape(N, -1), axis=1)
        yn = np.linalg.norm(Yn.reshape(N, -1), axis=1)
        bound = 3 * vh * 2.0 ** -53 * np.outer(xn, yn)
        assert (np.abs(K - Kref) <= 4 * bound).all(), call
        Kws = s.block_cdot(X, Y).cpu().numpy()
        assert (np.abs(K - Kws) <= 8 * bound).all(), call


def test_noalloc_cdot_allocates_nothing():
    """The entry point's defining property: its calls take no device memory
    (torch's allocator and the driver's free-memory count are unchanged; the
    output K is allocated by the caller beforehand).  Measured after one
    first call, because that call looks up the scratch array's address and
    with CUDA's lazy module loading this is when the runtime loads the
    library's device image, which holds the array; that load is the
    runtime's, not an allocation by the entry point."""
    torch = gh.torch_mod()
    gh.ensure_built()
    from paper_1710_09745_gb300 import load_library
    lib = load_library()
    dims = (8, 8, 8, 8)
    N = 8
    X = torch.as_tensor(hi.gaussian_sources(dims, N, seed=11)).cuda()
    Y = torch.as_tensor(hi.gaussian_sources(dims, N, seed=12)).cuda()
    K = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()

    def call():
        return lib.blockcg_block_cdot_noalloc(ct.c_void_p(X.data_ptr()), ct.c_void_p(Y.data_ptr()),
                                              N, X.shape[1], ct.c_void_p(K.data_ptr()),
                                              ct.c_void_p(stream.cuda_stream))
    assert call() == 0
    import gc
    gc.collect()  # tensors left by earlier tests are freed now, not during the measurement
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert call() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() <= alloc0
    assert free1 >= free0
    Kref = oblock.block_cdot(oblock.as_columns(X.cpu().numpy()), oblock.as_columns(Y.cpu().numpy()))
    assert np.abs(K.cpu().numpy() - Kref).max() < 1e-9


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
