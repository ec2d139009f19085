"""GPU: batches of uneven problems (batched launches, CUDA graph), the tuner's layouts.

A batch runs each problem's own plan arithmetic: its forward results must equal those of
single plans exactly.  The batched adjoint splits each class's rank sum over its own
number of CTAs, so it agrees with single plans to FP32 rounding (2-norm 1e-6).  Each
problem is also checked against the oracle (the low-rank
oracle on the grid the plan chose, at the tolerances of test_gpu_nufft.py, and the
direct sum of eq. (1.2) at eps for a few rows).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import direct, lowrank  # noqa: E402
from paper_1701_04492_gb300 import workloads as wl  # noqa: E402
from parity import assert_close  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1701_04492_gb300 import api as a
    return a


def _rel2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


TOL_REL = {"f32": 1e-5, "f64": 1e-13}
CDT = {"f32": torch.complex64, "f64": torch.complex128}
NPC = {"f32": np.complex64, "f64": np.complex128}


def _problems(count, seed, lo=10, hi=15):
    """Uneven sizes (non-powers of two), mixed eps, uniform samples; one empty problem."""
    N, eps = wl.uneven_batch(count, seed, lo, hi)
    r = np.random.default_rng(seed)
    M = [int(n * f) for n, f in zip(N, r.uniform(0.5, 1.5, count))]
    M[count // 2] = 0
    xs = [wl.samples_uniform(m, seed + 100 + i) for i, m in enumerate(M)]
    return [int(n) for n in N], xs, eps


def _packed(prec, N, seed):
    c = wl.coeffs_cn(int(sum(N)), seed).astype(NPC[prec])
    return torch.tensor(c, device="cuda"), c.astype(np.complex128)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_forward_matches_single_plans_and_oracle(api, prec):
    N, xs, eps = _problems(20, 11)
    b = api.Batch(N, xs, eps, prec)
    c_dev, c = _packed(prec, N, 5)
    f = b.forward(c_dev).cpu().numpy()
    for i in range(b.count):
        n0, n1 = b.offN[i], b.offN[i + 1]
        m0, m1 = b.offM[i], b.offM[i + 1]
        p = api.Plan(N[i], xs[i], eps[i], prec)
        assert p.L == b.L[i] and p.K == b.K[i]
        if m1 == m0:
            continue
        fi = p.forward(c_dev[n0:n1].contiguous()).cpu().numpy()
        assert np.array_equal(f[m0:m1], fi), i        # the same arithmetic, bit for bit
        P = lowrank.plan(N[i], xs[i], eps[i], int(b.L[i]))
        fo = lowrank.nufft2(P, c[n0:n1])
        assert_close(f[m0:m1], fo, prec, what=str(i))
        rows = np.arange(0, m1 - m0, max(1, (m1 - m0) // 16))
        fd = direct.nudft2(xs[i][rows], c[n0:n1])
        bound = max(eps[i], 5e-6 if prec == "f32" else 1e-13) * np.sum(np.abs(c[n0:n1]))
        assert np.max(np.abs(f[m0:m1][rows] - fd)) <= bound, i


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_adjoint_matches_single_plans_and_oracle(api, prec):
    N, xs, eps = _problems(16, 12)
    b = api.Batch(N, xs, eps, prec)
    g = wl.cotangent_cn(int(b.total_M), 6).astype(NPC[prec])
    g_dev = torch.tensor(g, device="cuda")
    cc = b.adjoint(g_dev).cpu().numpy()
    for i in range(b.count):
        n0, n1 = b.offN[i], b.offN[i + 1]
        m0, m1 = b.offM[i], b.offM[i + 1]
        if m1 == m0:
            assert np.all(cc[n0:n1] == 0)
            continue
        p = api.Plan(N[i], xs[i], eps[i], prec)
        ci = p.adjoint(g_dev[m0:m1].contiguous()).cpu().numpy()
        if prec == "f64":
            assert np.array_equal(cc[n0:n1], ci), i      # FP64 batches run each plan's launches
        else:
            assert _rel2(cc[n0:n1], ci) <= 1e-6, i
        P = lowrank.plan(N[i], xs[i], eps[i], int(b.L[i]))
        co = lowrank.nufft2_adjoint(P, g[m0:m1].astype(np.complex128))
        assert_close(cc[n0:n1], co, prec, what=str(i))


def test_batch_each_and_per_problem_match_batched(api):
    N, xs, eps = _problems(24, 13)
    b = api.Batch(N, xs, eps, "f32")
    bp = api.Batch(N, xs, eps, "f32", per_problem=True)
    assert bp.classes == b.count and b.classes < b.count
    c_dev, _ = _packed("f32", N, 7)
    f = b.forward(c_dev)
    assert torch.equal(b.forward_each(c_dev), f)
    assert torch.equal(bp.forward(c_dev), f)
    g_dev = torch.tensor(wl.cotangent_cn(int(b.total_M), 8).astype(np.complex64), device="cuda")
    ca = b.adjoint(g_dev).cpu().numpy()
    ce = b.adjoint_each(g_dev)
    assert torch.equal(bp.adjoint(g_dev), ce)          # both run each plan's own launches
    assert _rel2(ce.cpu().numpy(), ca) <= 1e-6
    b.check()


@pytest.mark.parametrize("per_problem", [False, True])
def test_batch_graph_replay_matches_eager(api, per_problem):
    N, xs, eps = _problems(24, 14)
    eager = api.Batch(N, xs, eps, "f32", per_problem=per_problem)
    gb = api.Batch(N, xs, eps, "f32", graph=True, per_problem=per_problem)
    c_dev, _ = _packed("f32", N, 9)
    g_dev = torch.tensor(wl.cotangent_cn(int(gb.total_M), 10).astype(np.complex64), device="cuda")
    ref_f, ref_c = eager.forward(c_dev), eager.adjoint(g_dev)
    f = torch.empty_like(ref_f)
    cc = torch.empty_like(ref_c)
    for it in range(4):        # eager, capture + replay, replay, replay
        f.fill_(0)
        cc.fill_(0)
        gb.forward(c_dev, f)
        gb.adjoint(g_dev, cc)
        torch.cuda.synchronize()
        assert torch.equal(f, ref_f), it
        assert torch.equal(cc, ref_c), it
    # other pointers: direct launches again, then a new graph
    f2 = torch.empty_like(ref_f)
    for it in range(3):
        gb.forward(c_dev, f2)
        assert torch.equal(f2, ref_f), it
    gb.check()


def test_batch_large_problem_runs_its_own_launches(api):
    """A grid beyond 2^18 points (N = 300000 -> L = 2^19) joins an FP32 batch."""
    N = [1500, 300000, 5000]
    xs = [wl.samples_uniform(m, 20 + i) for i, m in enumerate([1700, 250000, 4000])]
    eps = [1e-7, 1e-9, 1e-4]
    b = api.Batch(N, xs, eps, "f32")
    assert b.L[1] == 1 << 19 and b.classes == 3
    c_dev, c = _packed("f32", N, 21)
    f = b.forward(c_dev).cpu().numpy()
    for i in range(3):
        p = api.Plan(N[i], xs[i], eps[i], "f32")
        fi = p.forward(c_dev[b.offN[i]:b.offN[i + 1]].contiguous()).cpu().numpy()
        assert np.array_equal(f[b.offM[i]:b.offM[i + 1]], fi), i


def test_batch_c5_shape_against_oracle_sample(api):
    """The serving workload's shape: 512 problems, N log-uniform in [2^10, 2^18],
    eps in {1e-4, 1e-7, 1e-12}, uniform x, M = N.  Every problem's first rows are
    checked against the direct sum at its eps (FP32 floor 5e-6)."""
    N, eps = wl.uneven_batch(512, 2024)
    xs = [wl.samples_uniform(int(n), 3000 + i) for i, n in enumerate(N)]
    b = api.Batch([int(n) for n in N], xs, eps, "f32", graph=True)
    c_dev, c = _packed("f32", N, 31)
    f = torch.empty(b.total_M, dtype=torch.complex64, device="cuda")
    for _ in range(3):
        b.forward(c_dev, f)
    f = f.cpu().numpy()
    ref = api.Batch([int(n) for n in N], xs, eps, "f32", per_problem=True).forward(c_dev).cpu().numpy()
    assert np.array_equal(f, ref)
    for i in range(0, 512, 37):
        n0, n1, m0 = b.offN[i], b.offN[i + 1], b.offM[i]
        rows = np.arange(8)
        fd = direct.nudft2(xs[i][rows], c[n0:n1])
        bound = max(eps[i], 5e-6) * np.sum(np.abs(c[n0:n1]))
        assert np.max(np.abs(f[m0 + rows] - fd)) <= bound, i


# ---- layouts the tuner explores ------------------------------------------------------

@pytest.mark.parametrize("N", [2048, 3000, 1 << 15])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_long_columns_split_matches_oracle(api, N, prec):
    """The other four-step split of an odd log2 L (L2 = 2 L1) computes the same transform."""
    x = wl.samples_uniform(N, 40)
    L = 1024
    while L < N:
        L *= 2
    if (L.bit_length() - 1) % 2 == 0:
        L *= 2          # an odd log2 L, so that the split differs
    p = api.Plan(N, x, 1e-9, prec, L=L, long_columns=True)
    q = api.Plan(N, x, 1e-9, prec, L=L)
    c = wl.coeffs_cn(N, 41).astype(NPC[prec])
    c_dev = torch.tensor(c, device="cuda")
    f = p.forward(c_dev).cpu().numpy()
    P = lowrank.plan(N, x, 1e-9, L)
    fo = lowrank.nufft2(P, c.astype(np.complex128))
    assert_close(f, fo, prec, what="oracle")
    assert _rel2(f, q.forward(c_dev).cpu().numpy()) <= TOL_REL[prec]
    g = wl.cotangent_cn(N, 42).astype(NPC[prec])
    ca = p.adjoint(torch.tensor(g, device="cuda")).cpu().numpy()
    assert_close(ca, lowrank.nufft2_adjoint(P, g.astype(np.complex128)), prec, what="oracle")


@pytest.mark.parametrize("N,eps", [(1500, 1e-12), (5000, 1e-7), (40000, 1e-4), (1 << 16, 1e-9)])
def test_autotuned_plan_matches_oracle(api, N, eps):
    x = wl.samples_uniform(N, 50)
    p = api.Plan(N, x, eps, "f32", autotune=True)
    L0 = 1024
    while L0 < N:
        L0 *= 2
    assert p.L in (L0, 2 * L0)
    c = wl.coeffs_cn(N, 51).astype(np.complex64)
    f = p.forward(torch.tensor(c, device="cuda")).cpu().numpy()
    P = lowrank.plan(N, x, eps, p.L)
    assert P.K == p.K
    assert_close(f, lowrank.nufft2(P, c.astype(np.complex128)), "f32", what="oracle")
    # the cached choice: a second plan of the same shape takes the same layout
    p2 = api.Plan(N, wl.samples_uniform(N, 52), eps, "f32", autotune=True)
    assert p2.L == p.L


def test_tune_table_carries_choices_to_a_cleared_process_table(api, tmp_path):
    """The tuner's choices written by nufft_tune_save and read back after a clear make
    a new autotuned plan take the stored layout; a hand-written choice (here: the
    oversampled grid) is taken as stored, without timing."""
    N, eps = 5000, 1e-7
    x = wl.samples_uniform(N, 53)
    p = api.Plan(N, x, eps, "f32", autotune=True)
    path = tmp_path / "tune.txt"
    assert api.tune_save(path) >= 1
    api.tune_clear()
    assert api.tune_load(path) >= 1
    assert api.Plan(N, wl.samples_uniform(N, 54), eps, "f32", autotune=True).L == p.L
    # a hand-written entry forcing the grid 2 L0 for another shape
    N2, M2 = 3000, 3000
    x2 = wl.samples_uniform(M2, 55)
    K0 = api.Plan(N2, x2, eps, "f32").K               # the rank on the default grid is the key
    Mb = 1
    while Mb < M2:
        Mb *= 2
    dev = torch.cuda.current_device()
    forced = tmp_path / "forced.txt"
    forced.write_text("nufft-tune-table 1\n%d %d %d %.17g 0 %d -> 8192 0 0\n" % (dev, N2, Mb, eps, K0))
    assert api.tune_load(forced) == 1
    q = api.Plan(N2, x2, eps, "f32", autotune=True)
    assert q.L == 8192
    c = wl.coeffs_cn(N2, 56).astype(np.complex64)
    f = q.forward(torch.tensor(c, device="cuda")).cpu().numpy()
    P = lowrank.plan(N2, x2, eps, 8192)
    assert_close(f, lowrank.nufft2(P, c.astype(np.complex128)), "f32", what="oracle")
    api.tune_clear()


def test_batch_autotuned_matches_oracle(api):
    """The batch tuner may move a class to the grid 2 L0 or the other split; every
    problem still computes its transform (low-rank oracle on the grid it got)."""
    N, xs, eps = _problems(40, 15, lo=10, hi=14)
    b = api.Batch(N, xs, eps, "f32", autotune=True)
    c_dev, c = _packed("f32", N, 16)
    f = b.forward(c_dev).cpu().numpy()
    g = wl.cotangent_cn(int(b.total_M), 17).astype(np.complex64)
    cc = b.adjoint(torch.tensor(g, device="cuda")).cpu().numpy()
    for i in range(b.count):
        n0, n1 = b.offN[i], b.offN[i + 1]
        m0, m1 = b.offM[i], b.offM[i + 1]
        L0 = max(1024, 1 << (N[i] - 1).bit_length())
        assert b.L[i] in (L0, 2 * L0)
        if m1 == m0:
            continue
        P = lowrank.plan(N[i], xs[i], eps[i], int(b.L[i]))
        assert P.K == b.K[i]
        assert_close(f[m0:m1], lowrank.nufft2(P, c[n0:n1]), "f32", what=str(i))
        assert_close(cc[n0:n1], lowrank.nufft2_adjoint(P, g[m0:m1].astype(np.complex128)), "f32", what=str(i))


@pytest.mark.parametrize("N,long_cols", [(2048, False), (3000, True), (1 << 15, False), (1 << 17, True)])
def test_half_tile_matches_oracle(api, N, long_cols):
    """The tuners' tile axis: the column pass with half the columns per CTA computes the
    same transform (forward and adjoint), alone and with the other four-step split."""
    x = wl.samples_uniform(N, 43)
    L = 1024
    while L < N:
        L *= 2
    if long_cols and (L.bit_length() - 1) % 2 == 0:
        L *= 2
    p = api.Plan(N, x, 1e-9, "f32", L=L, half_tile=True, long_columns=long_cols)
    c = wl.coeffs_cn(N, 44).astype(np.complex64)
    f = p.forward(torch.tensor(c, device="cuda")).cpu().numpy()
    P = lowrank.plan(N, x, 1e-9, L)
    assert_close(f, lowrank.nufft2(P, c.astype(np.complex128)), "f32", what="oracle")
    g = wl.cotangent_cn(N, 45).astype(np.complex64)
    ca = p.adjoint(torch.tensor(g, device="cuda")).cpu().numpy()
    assert_close(ca, lowrank.nufft2_adjoint(P, g.astype(np.complex128)), "f32", what="oracle")


def test_reserved_batch_calls_allocate_nothing_and_capture_in_a_graph(api):
    """After nufft2_plan_reserve the batch calls and the host-buffer step neither allocate
    nor synchronise: a batch bigger than the reservation is refused (NUFFT_ESTATE) instead
    of growing the workspace, and the very first batch forward, adjoint and forward-with-f'
    of a fresh plan can be captured into a CUDA graph whose replay equals the direct calls."""
    import ctypes
    from paper_1701_04492_gb300 import _lib
    lib = _lib.load()
    N, M, B = 4096, 5000, 5
    x = wl.samples_uniform(M, 900)
    plan = api.Plan(N, x, 1e-9, "f32")
    c = torch.tensor(np.stack([wl.coeffs_cn(N, 901 + b) for b in range(B)]).astype(np.complex64), device="cuda")
    g = torch.tensor(np.stack([wl.cotangent_cn(M, 911 + b) for b in range(B)]).astype(np.complex64), device="cuda")
    f = torch.empty(B, M, dtype=torch.complex64, device="cuda")
    fp = torch.empty_like(f)
    gc = torch.empty(B, N, dtype=torch.complex64, device="cuda")
    st = api._stream(plan.device)
    vp = ctypes.c_void_p
    # nothing reserved yet: the batched path refuses rather than allocating
    assert lib.nufft2_exec_batch(plan._h, B, vp(c.data_ptr()), N, vp(f.data_ptr()), M, st) == -5
    plan.reserve(B)
    assert lib.nufft2_exec_batch(plan._h, B + 1, vp(c.data_ptr()), N, vp(f.data_ptr()), M, st) == -5
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.forward_batch(c, f)
        plan.adjoint_batch(g, gc)
    torch.cuda.synchronize()
    f.zero_()
    gc.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(f, plan.forward_batch(c))
    assert torch.equal(gc, plan.adjoint_batch(g))
    # the forward with f', captured on its own (first use of that argument set)
    f2, fp2 = torch.empty_like(f), torch.empty_like(f)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s):
        plan.forward_deriv_batch(c, f2, fp2)
    g2.replay()
    torch.cuda.synchronize()
    fr, fpr = plan.forward_deriv_batch(c)
    assert torch.equal(f2, fr) and torch.equal(fp2, fpr)
    plan.check()


def test_step_host_needs_its_reservation(api):
    """nufft2_step_host without NUFFT_RESERVE_STEP_HOST returns NUFFT_ESTATE (it never
    allocates); after the reservation it runs."""
    import ctypes
    from paper_1701_04492_gb300 import _lib
    lib = _lib.load()
    N, M = 2048, 3000
    plan = api.Plan(N, wl.samples_uniform(M, 920), 1e-9, "f32")
    ch = torch.tensor(wl.coeffs_cn(N, 921).astype(np.complex64)).pin_memory()
    gh = torch.tensor(wl.cotangent_cn(M, 922).astype(np.complex64)).pin_memory()
    fh = torch.empty(M, dtype=torch.complex64).pin_memory()
    gch = torch.empty(N, dtype=torch.complex64).pin_memory()
    gxh = torch.empty(M, dtype=torch.float32).pin_memory()
    vp = ctypes.c_void_p
    args = [vp(t.data_ptr()) for t in (ch, gh, fh, gch, gxh)]
    assert lib.nufft2_step_host(plan._h, *args, api._stream(plan.device)) == -5
    plan.reserve(0, step_host=True)
    assert lib.nufft2_step_host(plan._h, *args, api._stream(plan.device)) == 0
    torch.cuda.synchronize()
    assert torch.equal(fh, plan.forward_deriv(ch.cuda())[0].cpu())   # the step's f comes with f'


@pytest.mark.parametrize("graph", [False, True])
def test_persistent_launch_matches_class_launches(api, graph):
    """NUFFT_BATCH_PERSISTENT: one launch per direction for every batched class (grids from
    2^10 to 2^15 points, several rank bounds, one empty problem).  The adjoint equals the
    class launches bit for bit; the forward agrees to FP32 rounding (its rank groups are
    re-chosen so that two CTAs fit per SM, and a group boundary moves where the compensated
    rank-sum folds in its correction); repeated calls give the same bits (the kernel resets
    its own ticket and counters), with and without a CUDA graph; and both agree with the
    oracle."""
    N, xs, eps = _problems(40, 31, lo=10, hi=15)
    ref = api.Batch(N, xs, eps, "f32")
    per = api.Batch(N, xs, eps, "f32", persistent=True, graph=graph)
    assert ref.launches_per_direction == 2 * ref.classes and ref.classes > 4
    assert per.launches_per_direction == 1
    c_dev, c = _packed("f32", N, 32)
    g = wl.cotangent_cn(int(ref.total_M), 33).astype(np.complex64)
    g_dev = torch.tensor(g, device="cuda")
    f0 = ref.forward(c_dev)
    a0 = ref.adjoint(g_dev)
    first = None
    for _ in range(3):
        f1 = per.forward(c_dev)
        a1 = per.adjoint(g_dev)
        torch.cuda.synchronize()
        assert _rel2(f1.cpu().numpy(), f0.cpu().numpy()) <= 1e-6
        assert torch.equal(a1, a0)
        if first is None:
            first = f1.clone()
        assert torch.equal(f1, first)
    per.check()
    fh = f1.cpu().numpy()
    for i in (0, len(N) // 3, len(N) - 1):
        m0, m1 = per.offM[i], per.offM[i + 1]
        n0, n1 = per.offN[i], per.offN[i + 1]
        if m1 == m0:
            continue
        P = lowrank.plan(N[i], xs[i], eps[i], int(per.L[i]))
        assert_close(fh[m0:m1], lowrank.nufft2(P, c[n0:n1]), "f32", what=str(i))
