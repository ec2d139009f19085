"""GPU: failure detection without a GPU fault.

Failures are injected on the host (an allocation reported as out of memory) or made by
a bounded device wait on an mbarrier that nothing completes; each must come back as a
status code, and the library and the CUDA context must stay usable afterwards.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lowrank  # noqa: E402
from paper_1701_04492_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1701_04492_gb300 import api as a
    return a


@pytest.fixture()
def lib():
    from paper_1701_04492_gb300 import _lib
    lb = _lib.load()
    yield lb
    lb.nufft_test_fail_alloc(-1)


def _works(api, N=4096):
    x = wl.samples_uniform(N, 60)
    c = wl.coeffs_cn(N, 61).astype(np.complex64)
    p = api.Plan(N, x, 1e-6, "f32")
    f = p.forward(torch.tensor(c, device="cuda")).cpu().numpy()
    P = lowrank.plan(N, x, 1e-6, p.L)
    fo = lowrank.nufft2(P, c.astype(np.complex128))
    assert np.linalg.norm(f - fo) / np.linalg.norm(fo) <= 1e-5


@pytest.mark.parametrize("after", [0, 1, 5, 12])
def test_plan_allocation_failure_is_enomem(api, lib, after):
    from paper_1701_04492_gb300._lib import NufftError
    x = wl.samples_uniform(5000, 62)
    lib.nufft_test_fail_alloc(after)
    with pytest.raises(NufftError) as e:
        api.Plan(4096, x, 1e-9, "f32")
    assert e.value.code == -2
    lib.nufft_test_fail_alloc(-1)
    _works(api)


def test_batch_and_inverse_allocation_failures(api, lib):
    from paper_1701_04492_gb300._lib import NufftError
    N, eps = [1500, 3000, 7000], [1e-6, 1e-9, 1e-4]
    xs = [wl.samples_uniform(n, 63 + i) for i, n in enumerate(N)]
    lib.nufft_test_fail_alloc(40)          # a later plan of the batch
    with pytest.raises(NufftError) as e:
        api.Batch(N, xs, eps, "f32")
    assert e.value.code == -2
    lib.nufft_test_fail_alloc(-1)
    b = api.Batch(N, xs, eps, "f32")
    b.forward(torch.zeros(b.total_N, dtype=torch.complex64, device="cuda"))
    b.check()
    # the inverse's solver state: a failed build leaves the plan usable and a later call builds it
    M = 2048
    x = wl.samples_perturbed(M, 64, 1 / 8)
    p = api.Plan(M, x, 1e-12, "f64")
    f = p.forward(torch.tensor(wl.coeffs_cn(M, 65), device="cuda"))
    lib.nufft_test_fail_alloc(3)
    with pytest.raises(NufftError) as e:
        p.inverse(f)
    assert e.value.code == -2
    lib.nufft_test_fail_alloc(-1)
    c, it, rr = p.inverse(f, tol=1e-12)
    assert rr <= 1e-12 and it > 1
    _works(api)


def test_bounded_wait_times_out_and_context_survives(api, lib):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.nufft_test_wait_timeout(s) == -6       # NUFFT_ETIMEOUT after the 2 s limit
    torch.cuda.synchronize()
    _works(api)
