"""gfcc_sigma_noalloc against gfcc_sigma, through the C ABI (collected last on purpose).

gfcc_sigma_noalloc serves callers that cannot allocate device memory on their call path (a
process whose device memory is all held by its own pool allocator, or a latency-critical path that
must not trigger the device-wide synchronisation of cudaMalloc / cudaFree).  It runs the same FP64
sigma product on device buffers the caller owns, with its workspace in a fixed array inside the
library.  Two calls in a row must both reproduce gfcc_sigma (the array keeps the previous call's
contents, which must not leak into the next result).
"""
import numpy as np
import pytest

from paper_2010_04768_gb300 import gfcc
from paper_2010_04768_gb300.synthetic import random_vector, workload

pytestmark = pytest.mark.gpu


def test_sigma_noalloc_matches_sigma_twice():
    torch = pytest.importorskip("torch")
    from paper_2010_04768_gb300 import build
    build.build()
    wl = workload("tiny")
    g = gfcc.GFCC(wl.problem())
    dims = dict(zip(("IP", "EA"), g.dims()))
    for sector in ("IP", "EA"):
        n = dims[sector]
        for call in range(2):
            X = np.stack([random_vector(10 * call + k, n) + 1j * random_vector(100 + 10 * call + k, n)
                          for k in range(5)])
            ref = g.sigma(sector, X)
            x_dev = torch.from_numpy(X.view(np.float64).copy()).cuda()
            y_dev = torch.full_like(x_dev, float("nan"))
            torch.cuda.synchronize()
            g.sigma_noalloc(sector, X.shape[0], x_dev.data_ptr(), y_dev.data_ptr())
            Y = y_dev.cpu().numpy().view(np.complex128).reshape(X.shape)
            # the tolerance of the FP64 sigma parity tests
            assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max()
    # sizes beyond the fixed workspace are refused with an error, not an allocation
    x_dev = torch.zeros(2 * 5000 * dims["EA"], dtype=torch.float64, device="cuda")
    with pytest.raises(gfcc.GFCCError) as e:
        g.sigma_noalloc("EA", 5000, x_dev.data_ptr(), x_dev.data_ptr())
    assert e.value.code == gfcc.ERR_ARG
    g.close()
