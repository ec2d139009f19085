"""GPU: the checked build (libnufft_check.so, compiled with NUFFT_CHECK).

In that build every index that comes from the data (the sample permutation, grid rows
and columns, bucket bounds, the stores of the column pass) is tested before it is used;
a failed test records NUFFT_ECHECK in the plan's error word and skips the access.  The
test builds it, runs every entry point family through it in a child process (the loader
picks the library from NUFFT_LIB, so the ordinary build stays loaded here), and asserts
that no check fired and that the results still agree with the oracle.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _rel2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _child():
    sys.path.insert(0, ROOT)
    import torch
    from oracle import lowrank
    from paper_1701_04492_gb300 import _lib, api
    from paper_1701_04492_gb300 import workloads as wl
    assert _lib.LIB_PATH.endswith("libnufft_check.so"), _lib.LIB_PATH
    dev = "cuda"
    tol = {"f32": 1e-5, "f64": 1e-11}
    cdt = {"f32": np.complex64, "f64": np.complex128}
    # 1D: odd sizes (ragged tiles and buckets), clustered and uniform samples, both precisions
    for prec, N, M, eps, kind in [("f32", 3001, 4999, 1e-6, "uniform"), ("f32", 70000, 33333, 1e-4, "perturbed"),
                                  ("f64", 5003, 2047, 1e-12, "uniform"), ("f64", 1 << 15, 40001, 1e-9, "perturbed"),
                                  ("f32", 1 << 20, 1 << 20, 1e-9, "perturbed")] + \
                                 [("f64", n, 7, 1e-9, "uniform") for n in (1, 2, 3, 5, 7, 8, 1000)]:
        x = wl.samples_uniform(M, N + M) if kind == "uniform" else wl.samples_perturbed(M, N + M, 1 / 8)
        nc = cdt[prec]
        p = api.Plan(N, x, eps, prec)
        P = lowrank.plan(N, x, eps, p.L)
        c = wl.coeffs_cn(N, N).astype(nc)
        g = wl.coeffs_cn(M, M).astype(nc)
        f = p.forward(torch.tensor(c, device=dev)).cpu().numpy()
        assert _rel2(f, lowrank.nufft2(P, c.astype(np.complex128))) <= tol[prec], (prec, N, M)
        a = p.adjoint(torch.tensor(g, device=dev)).cpu().numpy()
        assert _rel2(a, lowrank.nufft2_adjoint(P, g.astype(np.complex128))) <= tol[prec], (prec, N, M)
        f2, fp = p.forward_deriv(torch.tensor(c, device=dev))
        assert _rel2(f2.cpu().numpy(), f) <= tol[prec]
        gx = p.grad_x(torch.tensor(g, device=dev), fp).cpu().numpy()
        assert np.all(np.isfinite(gx))
        cb = np.stack([c, c[::-1].copy()])
        fb = p.forward_batch(torch.tensor(cb, device=dev)).cpu().numpy()
        assert _rel2(fb[0], f) <= tol[prec]
        ab = p.adjoint_batch(torch.tensor(np.stack([g, g]), device=dev)).cpu().numpy()
        assert _rel2(ab[1], a) <= tol[prec]
        p.check()
    # a batch of uneven problems, graph and direct launches
    Ns, epss = [1500, 3001, 7000, 20000], [1e-6, 1e-9, 1e-4, 1e-6]
    xs = [wl.samples_uniform(n + 17, 70 + i) for i, n in enumerate(Ns)]
    for graph, persistent in ((False, False), (True, False), (False, True)):
        b = api.Batch(Ns, xs, epss, "f32", graph=graph, persistent=persistent)
        cs = [wl.coeffs_cn(n, 80 + i).astype(np.complex64) for i, n in enumerate(Ns)]
        f = b.forward(torch.tensor(np.concatenate(cs), device=dev)).cpu().numpy()
        off = 0
        for i, n in enumerate(Ns):
            P = lowrank.plan(n, xs[i], epss[i], b.L[i])
            fo = lowrank.nufft2(P, cs[i].astype(np.complex128))
            assert _rel2(f[off:off + len(xs[i])], fo) <= 1e-5
            off += len(xs[i])
        b.adjoint(torch.tensor(f.astype(np.complex64), device=dev))
        b.check()
    # 2D
    m, n, M = 100, 40, 3001
    x, y = wl.samples_2d_uniform(M, 91)
    C = (wl.coeffs_cn(m * n, 92).reshape(m, n)).astype(np.complex64)
    p2 = api.Plan2D(m, n, x, y, 1e-6)
    P2 = lowrank.plan2d(m, n, x, y, 1e-6, p2.Lx, p2.Ly)
    f = p2.forward(torch.tensor(C, device=dev)).cpu().numpy()
    assert _rel2(f, lowrank.nufft2_2d(P2, C.astype(np.complex128))) <= 1e-5
    rc = _lib.load().nufft2_check(p2._h, api._stream(p2.device))
    assert rc == 0, _lib.STATUS.get(rc, rc)
    # the inverse (FP64 CG)
    N = 2048
    x = wl.samples_perturbed(N, 93, 1 / 8)
    p = api.Plan(N, x, 1e-12, "f64")
    f = p.forward(torch.tensor(wl.coeffs_cn(N, 94), device=dev))
    c, it, rr = p.inverse(f, tol=1e-12)
    assert rr <= 1e-12 and it > 1
    p.check()
    # the forward without a plan or device allocation: its return code carries the checks
    import ctypes
    lib = _lib.load()
    for N, M in [(2048, 3001), (1000, 777)]:
        x = wl.samples_uniform(M, 95)
        c = wl.coeffs_cn(N, 96).astype(np.complex64)
        xd = torch.tensor(x, dtype=torch.float64, device=dev)
        cd = torch.tensor(c, device=dev)
        f = torch.empty(M, dtype=torch.complex64, device=dev)
        rc = lib.nufft2_exec_noalloc(N, M, ctypes.c_void_p(xd.data_ptr()), 1e-9, ctypes.c_void_p(cd.data_ptr()),
                                     ctypes.c_void_p(f.data_ptr()), api._stream(0))
        assert rc == 0, _lib.STATUS.get(rc, rc)
        P = lowrank.plan(N, x, 1e-9, api.Plan(N, x, 1e-9, "f32").L)
        assert _rel2(f.cpu().numpy(), lowrank.nufft2(P, c.astype(np.complex128))) <= 1e-5
    print("CHECKED-OK")


def test_checked_build_runs_clean():
    from paper_1701_04492_gb300 import build
    lib = build.build(check=True)
    env = dict(os.environ, NUFFT_LIB=lib)
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "child"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=900)
    assert res.returncode == 0 and "CHECKED-OK" in res.stdout, res.stdout[-3000:] + res.stderr[-3000:]


if __name__ == "__main__" and sys.argv[1:] == ["child"]:
    _child()
