"""RHQR-GMRES (Algorithm 8) on the GPU: the least-squares solution and the
update x = x0 + Q_m y of rhqr_arnoldi_solution against the oracle's
rhqr_gmres on the same sketch and operator, and a restarted solve of the
2-D convection-diffusion system to 1e-8."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import rhqr, sketch  # noqa: E402


@pytest.mark.parametrize("g,mmax,k", [(48, 30, 128), (40, 12, 64)])
def test_arnoldi_solution_matches_oracle_gmres(gpu_lib, g, mmax, k):
    from paper_2405_10923_gb300 import torch_api as ta

    n = g * g
    rng = np.random.default_rng(7)
    b = rng.standard_normal(n)
    x0 = 0.1 * rng.standard_normal(n)

    def A_np(v):
        return ri.stencil_apply(v.copy(), g)

    osk = sketch.SRHTSketch(n, k, 77)
    x_o, H_o, Q_o, h0_o = rhqr.rhqr_gmres(A_np, b, x0, osk, mmax)
    y_o = np.linalg.lstsq(H_o, h0_o, rcond=None)[0]

    sk = ta.Sketch(n, k, gpu_lib.SRHT, 77)
    arn = ta.Arnoldi(sk, n, mmax, dtype=torch.float64)
    bd = torch.tensor(b, device="cuda")
    xd = torch.tensor(x0, device="cuda")
    H = gpu_lib.colmajor(torch.zeros((mmax + 1, mmax), dtype=torch.float64, device="cuda"))
    h0, q = arn.begin(bd - ri.stencil_apply(xd.clone(), g))
    for j in range(mmax):
        h, q = arn.step(ri.stencil_apply(q.clone(), g))
        H[:, j] = h
    y, res, x = arn.solution(H, mmax, h0, x0=xd)
    torch.cuda.synchronize()
    assert ta.read_info(arn.info)["status"] == 0
    assert np.max(np.abs(H.cpu().numpy() - H_o)) <= 1e-10 * np.abs(H_o).max()
    assert np.max(np.abs(y.cpu().numpy() - y_o)) <= 1e-9 * max(1.0, np.abs(y_o).max())
    assert abs(float(res) - np.linalg.norm(h0_o - H_o @ y_o)) <= 1e-9 * np.linalg.norm(h0_o)
    assert np.max(np.abs(x.cpu().numpy() - x_o)) <= 1e-10 * max(1.0, np.abs(x_o).max())
    # sketched optimality (eq. rgmresopti): res is the sketched residual of x
    r = b - A_np(x.cpu().numpy())
    assert abs(np.linalg.norm(sketch.rh_sketch(r, mmax + 1, osk)) - float(res)) <= 1e-8 * np.linalg.norm(b)
    # y only (no update), and fewer steps than taken
    y2, res2, x2 = arn.solution(H, mmax - 3, h0)
    y2_o = np.linalg.lstsq(H_o[: mmax - 2, : mmax - 3], h0_o[: mmax - 2], rcond=None)[0]
    assert x2 is None
    assert np.max(np.abs(y2.cpu().numpy() - y2_o)) <= 1e-9 * max(1.0, np.abs(y2_o).max())
    with pytest.raises(gpu_lib.RHQRError):
        arn.solution(H, mmax + 1, h0)
    arn.close()
    sk.close()


def test_restarted_gmres_converges(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    g = 32
    n = g * g
    sk = ta.Sketch(n, 128, gpu_lib.SRHT, 5)
    b = torch.tensor(np.random.default_rng(3).standard_normal(n), device="cuda")
    solver = ta.GMRES(sk, n, restart=60)
    x, hist = solver.solve(lambda v: ri.stencil_apply(v.clone(), g), b, tol=1e-8, max_cycles=30)
    r = b - ri.stencil_apply(x.clone(), g)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(b)) <= 1e-8, hist
    assert hist[-1] < hist[0]
    solver.close()
    sk.close()


def test_arnoldi_solution_float32_basis(gpu_lib):
    """float32 basis: the same sketched least-squares problem, x within float32
    accuracy of the oracle's float64 cycle."""
    from paper_2405_10923_gb300 import torch_api as ta

    g, mmax, k = 40, 20, 64
    n = g * g
    rng = np.random.default_rng(9)
    b = rng.standard_normal(n)
    osk = sketch.SRHTSketch(n, k, 78)
    x_o, H_o, _, h0_o = rhqr.rhqr_gmres(lambda v: ri.stencil_apply(v.copy(), g), b, np.zeros(n), osk, mmax)
    sk = ta.Sketch(n, k, gpu_lib.SRHT, 78)
    arn = ta.Arnoldi(sk, n, mmax, dtype=torch.float32)
    bd = torch.tensor(b, dtype=torch.float32, device="cuda")
    H = gpu_lib.colmajor(torch.zeros((mmax + 1, mmax), dtype=torch.float64, device="cuda"))
    h0, q = arn.begin(bd)
    for j in range(mmax):
        h, q = arn.step(ri.stencil_apply(q.clone(), g))
        H[:, j] = h
    y, res, x = arn.solution(H, mmax, h0, x0=torch.zeros_like(bd))
    torch.cuda.synchronize()
    assert x.dtype == torch.float32
    assert np.max(np.abs(x.double().cpu().numpy() - x_o)) <= 1e-4 * np.abs(x_o).max()
    assert abs(float(res) - np.linalg.norm(h0_o - H_o @ np.linalg.lstsq(H_o, h0_o, rcond=None)[0])) \
        <= 1e-4 * np.linalg.norm(h0_o)
    arn.close()
    sk.close()


# ---------------------------------------------------------------------------
# the workload's operator in the library, and several right-hand sides at once
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_stencil_kernel_and_residual_match_definition(gpu_lib, dt):
    """rhqr_stencil_apply / rhqr_stencil_residual against the operator's
    definition (rhqr_inputs.stencil_apply in float64 numpy), 3 right-hand sides,
    a grid whose side is not a multiple of the block size."""
    from paper_2405_10923_gb300 import torch_api as ta

    g, nrhs = 37, 3
    n = g * g
    rng = np.random.default_rng(11)
    X = rng.standard_normal((n, nrhs))
    B = rng.standard_normal((n, nrhs))
    Xd = ta.block(n, nrhs, dt).copy_(torch.tensor(X, dtype=dt))
    Bd = ta.block(n, nrhs, dt).copy_(torch.tensor(B, dtype=dt))
    Xr, Br = Xd.double().cpu().numpy(), Bd.double().cpu().numpy()
    op = ta.StencilOperator(g, nrhs=nrhs)
    Y = op(Xd).double().cpu().numpy()
    want = np.stack([ri.stencil_apply(Xr[:, b].copy(), g) for b in range(nrhs)], axis=1)
    tol = 1e-14 if dt == torch.float64 else 1e-6
    assert np.max(np.abs(Y - want)) <= tol * np.abs(want).max()
    R, rn, bn = op.residual(Bd, Xd)
    Rw = Br - want
    assert np.max(np.abs(R.double().cpu().numpy() - Rw)) <= tol * np.abs(Rw).max()
    # the norms are those of the float64 residual, before it is stored in R's dtype
    assert np.allclose(rn.cpu().numpy(), np.linalg.norm(Rw, axis=0), rtol=1e-12)
    assert np.allclose(bn.cpu().numpy(), np.linalg.norm(Br, axis=0), rtol=1e-12)


def test_batched_arnoldi_matches_oracle_per_right_hand_side(gpu_lib):
    """nrhs = 4 processes in one handle (every kernel launched once per step for
    all of them): each process's H, y, x equal the oracle's rhqr_gmres on its
    own right-hand side and x0, with the library's stencil operator."""
    from paper_2405_10923_gb300 import torch_api as ta

    g, mmax, k, nrhs = 40, 16, 64, 4
    n = g * g
    rng = np.random.default_rng(12)
    Bm = rng.standard_normal((n, nrhs))
    X0 = 0.1 * rng.standard_normal((n, nrhs))
    osk = sketch.SRHTSketch(n, k, 79)
    sk = ta.Sketch(n, k, gpu_lib.SRHT, 79)
    op = ta.StencilOperator(g, nrhs=nrhs)
    arn = ta.Arnoldi(sk, n, mmax, dtype=torch.float64, nrhs=nrhs)
    Bd = ta.block(n, nrhs, torch.float64).copy_(torch.tensor(Bm))
    Xd = ta.block(n, nrhs, torch.float64).copy_(torch.tensor(X0))
    R, _, _ = op.residual(Bd, Xd)
    H = arn.hessenberg()
    h0, q = arn.begin(R)
    for j in range(mmax):
        h, q = arn.step(op(q))
        H[:, j, :] = h.t()
    y, res, x = arn.solution(H, mmax, h0, x0=Xd)
    torch.cuda.synchronize()
    assert ta.read_info(arn.info)["status"] == 0
    for b in range(nrhs):
        x_o, H_o, Q_o, h0_o = rhqr.rhqr_gmres(lambda v: ri.stencil_apply(v.copy(), g), Bm[:, b], X0[:, b], osk, mmax)
        y_o = np.linalg.lstsq(H_o, h0_o, rcond=None)[0]
        Hb = H[b].t().cpu().numpy()  # (mmax + 1) x mmax
        assert np.max(np.abs(Hb - H_o)) <= 1e-10 * np.abs(H_o).max()
        assert np.max(np.abs(y[:, b].cpu().numpy() - y_o)) <= 1e-9 * max(1.0, np.abs(y_o).max())
        assert abs(float(res[b]) - np.linalg.norm(h0_o - H_o @ y_o)) <= 1e-9 * np.linalg.norm(h0_o)
        assert np.max(np.abs(x[:, b].cpu().numpy() - x_o)) <= 1e-10 * max(1.0, np.abs(x_o).max())
    arn.close()
    sk.close()


def test_batched_restarted_gmres_converges(gpu_lib):
    """Restarted RHQR-GMRES on 8 right-hand sides of the 32 x 32 system with the
    library's operator and restart residual: every one reaches 1e-8."""
    from paper_2405_10923_gb300 import torch_api as ta

    g, nrhs = 32, 8
    n = g * g
    sk = ta.Sketch(n, 128, gpu_lib.SRHT, 6)
    op = ta.StencilOperator(g, nrhs=nrhs)
    B = ta.block(n, nrhs, torch.float64).copy_(torch.tensor(np.random.default_rng(4).standard_normal((n, nrhs))))
    solver = ta.GMRES(sk, n, restart=60, nrhs=nrhs)
    X, hist = solver.solve(op, B, tol=1e-8, max_cycles=30)
    R, rn, bn = op.residual(B, X)
    assert (rn.cpu().numpy() <= 1e-8 * bn.cpu().numpy()).all(), hist
    solver.close()
    sk.close()


def test_mixed_precision_restarted_gmres_converges(gpu_lib):
    """A float32 Krylov basis with a float64 iterate and float64 restart
    residual (the library's residual kernel and rhqr_arnoldi_solution_x) reaches
    1e-8 on 4 right-hand sides, which a float32 iterate could not."""
    from paper_2405_10923_gb300 import torch_api as ta

    g, nrhs = 32, 4
    n = g * g
    sk = ta.Sketch(n, 128, gpu_lib.SRHT, 7)
    op = ta.StencilOperator(g, nrhs=nrhs)
    B = ta.block(n, nrhs, torch.float64).copy_(torch.tensor(np.random.default_rng(5).standard_normal((n, nrhs))))
    solver = ta.GMRES(sk, n, restart=60, dtype=torch.float32, nrhs=nrhs)
    X, hist = solver.solve(op, B, tol=1e-8, max_cycles=40)
    assert X.dtype == torch.float64
    R, rn, bn = op.residual(B, X)
    assert (rn.cpu().numpy() <= 1e-8 * bn.cpu().numpy()).all(), hist
    solver.close()
    sk.close()
