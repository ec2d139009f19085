"""nufft2_exec_noalloc: the forward transform for callers that cannot allocate
device memory (it keeps its intermediates in one fixed array compiled into the
library).  Collected last on purpose: a failure here stops a -x run only after every
other test has run.  Its output must match the planned path (nufft2_plan +
nufft2_exec) within the FP32 tolerance of the parity tests, on two calls in a row
(the second reuses the fixed array the first one left behind)."""

import ctypes

import numpy as np
import pytest

from paper_1701_04492_gb300 import _lib, build
from paper_1701_04492_gb300 import workloads as wl

TOL_F32 = 1e-5   # ||df||_2 / ||f||_2, as for the FP32 parity tests


def test_rejects_sizes_beyond_the_fixed_array():
    build.build()
    lib = _lib.load()
    big = 65536 + 1
    # size checks come before any CUDA call
    assert lib.nufft2_exec_noalloc(big, 10, ctypes.c_void_p(1), 1e-9, ctypes.c_void_p(1), ctypes.c_void_p(1),
                                   None) == -4
    assert lib.nufft2_exec_noalloc(16, big, ctypes.c_void_p(1), 1e-9, ctypes.c_void_p(1),
                                   ctypes.c_void_p(1), None) == -4
    assert lib.nufft2_exec_noalloc(16, 10, None, 1e-9, ctypes.c_void_p(1), ctypes.c_void_p(1), None) == -1


@pytest.mark.gpu
# odd log2 L (2048, 32768) splits the grid into rows and columns of different lengths,
# with their own stage tables; "equispaced" is x_j = j/N, gamma = 0 and K = 1
@pytest.mark.parametrize("N,M,kind,eps", [(4096, 5000, "uniform", 1e-9), (65536, 65536, "perturbed", 1e-6),
                                          (1000, 777, "uniform", 1e-12), (3, 9, "uniform", 1e-4),
                                          (2048, 3001, "uniform", 1e-9), (32768, 40000, "perturbed", 1e-12),
                                          (4096, 4096, "equispaced", 1e-9)])
def test_matches_planned_path_twice(N, M, kind, eps):
    torch = pytest.importorskip("torch")
    from oracle import lowrank
    from paper_1701_04492_gb300.api import Plan
    lib = _lib.load()
    x = {"uniform": lambda: wl.samples_uniform(M, 77), "perturbed": lambda: wl.samples_perturbed(M, 77, 0.5),
         "equispaced": lambda: wl.samples_equispaced(N)}[kind]()
    c = wl.coeffs_cn(N, 77).astype(np.complex64)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    cd = torch.tensor(c, device="cuda")
    plan = Plan(N, x, eps, "f32")
    ref = plan.forward(cd).cpu().numpy()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        f = torch.full((M,), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
        rc = lib.nufft2_exec_noalloc(N, M, ctypes.c_void_p(xd.data_ptr()), eps, ctypes.c_void_p(cd.data_ptr()),
                                     ctypes.c_void_p(f.data_ptr()), stream)
        assert rc == 0, rc
        got = f.cpu().numpy()
        assert np.linalg.norm(got - ref) <= TOL_F32 * np.linalg.norm(ref)
    P = lowrank.plan(N, x, eps, plan.L)
    fo = lowrank.nufft2(P, c.astype(np.complex128))
    assert np.linalg.norm(got - fo) <= TOL_F32 * np.linalg.norm(fo)
    if kind == "equispaced":
        assert P.K == 1 and plan.K == 1
        assert np.linalg.norm(got - np.fft.fft(c.astype(np.complex128))) <= TOL_F32 * np.linalg.norm(fo)
