"""FP64 residual check of the GEMM on the GPU (Freivalds 1977) through the C ABI.

gao_gemm_residual / prog_gemm_residual evaluate, in binary64 on the device,
    r = C x - beta C0 x - alpha A (B x)   and   s = y^T C - beta y^T C0 - alpha (y^T A) B
and their norms against the reference sides.  The checks here:
  * on ragged small shapes (K = 0, a missing C0, shapes that are not multiples of 4),
    the device's r and s equal numpy's binary64 evaluation of the same formulas within
    binary64 rounding;
  * at n = 8192 on the BF16X6 GEMM program, the device residuals agree with the host
    Freivalds residual computed from the oracle's own copies of A, B, C0 (counter hash,
    binary64), and both sit under the 1e-6 gate;
  * one entry of C planted wrong by 1e-6 max|C| moves r in exactly one row and s in
    exactly one column, by that error times the sign vector's entry -- and nothing else.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    return g


def host_sides(A, B, C0, C, alpha, beta, x, y):
    """r, s, f, g of the right and left forms in binary64 (numpy)."""
    A, B, C = (np.asarray(t, dtype=np.float64) for t in (A, B, C))
    c0x = np.zeros(C.shape[0]) if C0 is None else np.asarray(C0, dtype=np.float64) @ x
    yc0 = np.zeros(C.shape[1]) if C0 is None else y @ np.asarray(C0, dtype=np.float64)
    b = 0.0 if C0 is None else beta
    abx = A @ (B @ x)
    yab = (y @ A) @ B
    return C @ x - b * c0x - alpha * abx, y @ C - b * yc0 - alpha * yab, alpha * abx + b * c0x, alpha * yab + b * yc0


def device_residual(gao, torch, A, B, C0, C, alpha, beta, x, y):
    M, N = C.shape
    K = A.shape[1]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    tA, tB, tC = dev(A.astype(np.float32)), dev(B.astype(np.float32)), dev(C.astype(np.float32))
    tC0 = dev(C0.astype(np.float32)) if C0 is not None else None
    tx, ty = dev(x), dev(y)
    nb = gao.gao_gemm_residual_scratch(M, N, K)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    rv = torch.empty(M, dtype=torch.float64, device="cuda")
    sv = torch.empty(N, dtype=torch.float64, device="cuda")
    ptr = lambda t: 0 if (t is None or t.numel() == 0) else t.data_ptr()
    torch.cuda.synchronize()
    res = gao.gao_gemm_residual(ptr(tA), ptr(tB), ptr(tC0), ptr(tC), M, N, K, alpha, beta, ptr(tx), ptr(ty),
                                scratch.data_ptr(), nb, rv.data_ptr(), sv.data_ptr())
    return res, rv.cpu().numpy(), sv.cpu().numpy()


@pytest.mark.parametrize("M,N,K,with_c0", [(129, 77, 33, True), (1, 1, 1, True), (257, 131, 0, True),
                                           (64, 1030, 517, False), (2000, 3, 7, True), (5, 4097, 64, True)])
def test_residual_matches_numpy_binary64(gao, M, N, K, with_c0):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.uniform(-1, 1, (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (K, N)).astype(np.float32)
    C0 = rng.uniform(-1, 1, (M, N)).astype(np.float32) if with_c0 else None
    alpha, beta = 1.5, 0.5
    exact = alpha * (A.astype(np.float64) @ B.astype(np.float64))
    if with_c0:
        exact += beta * C0.astype(np.float64)
    C = (exact * (1.0 + 1e-6 * rng.standard_normal((M, N)))).astype(np.float32)  # a result with small errors
    x, y = rng.choice([-1.0, 1.0], N), rng.choice([-1.0, 1.0], M)
    res, rv, sv = device_residual(gao, torch, A, B, C0, C, alpha, beta, x, y)
    r, s, f, g = host_sides(A, B, C0, C, alpha, beta, x, y)
    # every term is exact in binary64 up to the sums' rounding: |error| <= K u64 |terms|
    tol_r = 1e-13 * (np.abs(A).astype(np.float64) @ (np.abs(B).astype(np.float64) @ np.ones(N)) * alpha +
                     np.abs(C).astype(np.float64) @ np.ones(N) + (0 if C0 is None else np.abs(C0).sum(1))) + 1e-300
    assert np.all(np.abs(rv - r) <= tol_r + 1e-13 * np.abs(f).max())
    assert np.all(np.abs(sv - s) <= 1e-12 * (np.abs(g).max() + np.abs(C).sum(0)) + 1e-300)
    nr = np.linalg.norm(r) / np.linalg.norm(f)
    ns = np.linalg.norm(s) / np.linalg.norm(g)
    assert abs(res["right"] - nr) <= 1e-9 * nr + 1e-15
    assert abs(res["left"] - ns) <= 1e-9 * ns + 1e-15
    assert abs(res["right_inf"] - np.abs(r).max() / np.abs(f).max()) <= 1e-9 * res["right_inf"] + 1e-15
    assert abs(res["left_inf"] - np.abs(s).max() / np.abs(g).max()) <= 1e-9 * res["left_inf"] + 1e-15
    assert 0 <= res["right_argmax"] < M and 0 <= res["left_argmax"] < N
    assert abs(abs(rv[res["right_argmax"]]) - np.abs(rv).max()) == 0.0
    assert abs(abs(sv[res["left_argmax"]]) - np.abs(sv).max()) == 0.0


def test_residual_is_deterministic(gao):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    M, N, K = 300, 513, 200
    A, B, C0 = (rng.uniform(-1, 1, s).astype(np.float32) for s in ((M, K), (K, N), (M, N)))
    C = (1.5 * A.astype(np.float64) @ B + 0.5 * C0).astype(np.float32)
    x, y = rng.choice([-1.0, 1.0], N), rng.choice([-1.0, 1.0], M)
    a = device_residual(gao, torch, A, B, C0, C, 1.5, 0.5, x, y)
    b = device_residual(gao, torch, A, B, C0, C, 1.5, 0.5, x, y)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.fixture(scope="module")
def n8192_run(gao):
    """The n = 8192 GEMM program (BF16X6, all on the GPU), C0 kept in a buffer of its own."""
    n, seed = 8192, W.SEED_N8192
    prog = W.gemm_only(n, seed)
    p = gao.prog_from_workload(prog, gemm_prec=gao.BF16X6)
    gao.prog_run(p, 0b11)
    C = gao.prog_output(p, prog.index("C"))
    yield gao, prog, p, C
    gao.prog_destroy(p)


def test_n8192_device_residual_agrees_with_host_freivalds(n8192_run):
    gao, prog, p, C = n8192_run
    n, seed = 8192, prog.seed
    rng = np.random.default_rng(8192)
    x, y = rng.choice([-1.0, 1.0], n), rng.choice([-1.0, 1.0], n)
    dev = gao.prog_gemm_residual(p, 1, x, y)
    A, B, C0 = (oracle.init_matrix(seed, b, n, n) for b in (0, 1, 2))
    r, s, f, g = host_sides(A, B, C0, C, 1.5, 0.5, x, y)
    right, left = np.linalg.norm(r) / np.linalg.norm(f), np.linalg.norm(s) / np.linalg.norm(g)
    print(f"n=8192 BF16X6 residual: device right {dev['right']:.4e} left {dev['left']:.4e}, "
          f"host right {right:.4e} left {left:.4e}")
    assert abs(dev["right"] - right) <= 1e-6 * right
    assert abs(dev["left"] - left) <= 1e-6 * left
    assert max(dev["right"], dev["left"]) <= 1e-6


def test_n8192_planted_entry_moves_one_row_and_one_column(n8192_run):
    torch = pytest.importorskip("torch")
    gao, prog, p, C = n8192_run
    n = 8192
    rng = np.random.default_rng(11)
    x, y = rng.choice([-1.0, 1.0], n), rng.choice([-1.0, 1.0], n)
    i, j = 5000, 1234
    delta = np.float32(1e-6 * float(np.abs(C).max()))
    Cp = C.copy()
    Cp[i, j] = np.float32(Cp[i, j] + delta)
    d = float(Cp[i, j]) - float(C[i, j])  # the planted error as stored in binary32
    assert d != 0.0
    ptr = lambda b: gao.prog_device_ptr(p, prog.index(b))
    nb = gao.gao_gemm_residual_scratch(n, n, n)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    tx, ty = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = {}
    for name, Cm in (("clean", C), ("planted", Cp)):
        tC = torch.from_numpy(Cm).cuda()
        rv = torch.empty(n, dtype=torch.float64, device="cuda")
        sv = torch.empty(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        res = gao.gao_gemm_residual(ptr("A"), ptr("B"), ptr("C0"), tC.data_ptr(), n, n, n, 1.5, 0.5, tx.data_ptr(),
                                    ty.data_ptr(), scratch.data_ptr(), nb, rv.data_ptr(), sv.data_ptr())
        out[name] = (res, rv.cpu().numpy(), sv.cpu().numpy())
    dr = out["planted"][1] - out["clean"][1]
    ds = out["planted"][2] - out["clean"][2]
    assert np.count_nonzero(dr) == 1 and np.count_nonzero(ds) == 1
    assert int(np.flatnonzero(dr)[0]) == i and int(np.flatnonzero(ds)[0]) == j
    assert abs(dr[i] - d * x[j]) <= 1e-6 * abs(d)
    assert abs(ds[j] - d * y[i]) <= 1e-6 * abs(d)
    # one 128 x 128 tile (1/4096 of C) off by 1e-3 relative: ~1.5e-5 normwise, far above the
    # rounding level of the clean result and over the 1e-6 gate
    Ct = C.copy()
    Ct[1024:1152, 2048:2176] *= np.float32(1.0 + 1e-3)
    res_t, _, _ = device_residual_on(gao, torch, ptr, Ct, n, x, y, scratch, nb)
    clean = max(out["clean"][0]["right"], out["clean"][0]["left"])
    assert min(res_t["right"], res_t["left"]) > max(10 * clean, 1e-6)


def device_residual_on(gao, torch, ptr, Cm, n, x, y, scratch, nb):
    tC = torch.from_numpy(Cm).cuda()
    tx, ty = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    torch.cuda.synchronize()
    res = gao.gao_gemm_residual(ptr("A"), ptr("B"), ptr("C0"), tC.data_ptr(), n, n, n, 1.5, 0.5, tx.data_ptr(),
                                ty.data_ptr(), scratch.data_ptr(), nb)
    return res, None, None


def test_prog_gemm_residual_rejects_in_place_gemm(gao):
    prog = W.six_loop(64, 3, outputs=("C",))  # C = alpha A B + beta C: C0 overwritten
    p = gao.prog_from_workload(prog, gemm_prec=gao.BF16X6)
    gao.prog_run(p, 0b111111)
    with pytest.raises(gao.GaoError):
        gao.prog_gemm_residual(p, 1, np.ones(64), np.ones(64))
    assert "C0" in gao.gao_last_error()
    with pytest.raises(gao.GaoError):
        gao.prog_gemm_residual(p, 0, np.ones(64), np.ones(64))  # loop 0 is the INIT
    gao.prog_destroy(p)


@pytest.mark.parametrize("prec", ["fp32_simt", "bf16x3"])
def test_prog_gemm_residual_small_programs(gao, prec):
    """prog_gemm_residual on a ragged program whose GEMM ran on the GPU and on the CPU: the
    device check agrees with numpy on the program's own outputs."""
    n, seed = 300, 41
    prog = W.gemm_only(n, seed)
    p = gao.prog_from_workload(prog, gemm_prec={"fp32_simt": gao.FP32_SIMT, "bf16x3": gao.BF16X3}[prec])
    rng = np.random.default_rng(2)
    x, y = rng.choice([-1.0, 1.0], n), rng.choice([-1.0, 1.0], n)
    A, B, C0 = (oracle.init_matrix(seed, b, n, n) for b in (0, 1, 2))
    for gene in (0b11, 0b01, 0b00):  # GEMM on the GPU; on the host (buffers copied up for the check)
        gao.prog_run(p, gene)
        C = gao.prog_output(p, prog.index("C"))
        dev = gao.prog_gemm_residual(p, 1, x, y)
        r, s, f, g = host_sides(A, B, C0, C, 1.5, 0.5, x, y)
        assert abs(dev["right"] - np.linalg.norm(r) / np.linalg.norm(f)) <= 1e-9 * dev["right"] + 1e-15
        assert abs(dev["left"] - np.linalg.norm(s) / np.linalg.norm(g)) <= 1e-9 * dev["left"] + 1e-15
        assert max(dev["right"], dev["left"]) <= (1e-6 if prec == "fp32_simt" else 2e-5)
    gao.prog_destroy(p)
