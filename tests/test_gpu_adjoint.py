"""Differentiation path on the GPU against the oracle: the transposed H-matvec,
the transposed (adjoint) solve, the potential at evaluation points and its
adjoint, and gradients of a potential misfit through the solve (dense oracle
gradient at level 4, central finite differences at level 6)."""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lvl4(orc):
    need_gpu()
    cfg = meshgen.config("differentiation4")
    g = GpuH(cfg["V"], cfg["T"], leaf=64, eta=1.5, eps=1e-10, kmax=64, factor_dtype=1, dense_dtype=1)
    yield g, cfg
    g.close()


def _exported_operator(orc, g, trans):
    perm = g.perm()
    ex = g.export()
    dl, al = g.leaves(True), g.leaves(False)

    def mv(x):
        ym = orc.hmatvec_raw(g.n, dl, ex["dense_off"], ex["dense"], al, ex["rank"], ex["u_off"], ex["w_off"],
                             ex["uw"], x[perm], trans=trans)
        y = np.empty(g.n)
        y[perm] = ym
        return y

    return mv


def test_transposed_matvec(orc, lvl4):
    g, _ = lvl4
    rng = np.random.default_rng(1)
    mvt = _exported_operator(orc, g, True)
    for _ in range(2):
        x, y = rng.standard_normal(g.n), rng.standard_normal(g.n)
        hx, hty = g.matvec(x), g.matvec(y, trans=1)
        # adjoint identity y.(H x) = x.(H^T y)
        assert abs(y @ hx - x @ hty) <= 1e-13 * np.linalg.norm(y) * np.linalg.norm(hx)
        # the oracle applying the exported operator transposed
        ref = mvt(y)
        assert np.linalg.norm(hty - ref) <= 1e-12 * np.linalg.norm(ref)
        # FP32 copy, transposed
        hty32 = g.matvec(y, trans=1, prec=1)
        assert np.linalg.norm(hty32 - hty) <= 1e-5 * np.linalg.norm(hty)


def test_transposed_solve(orc, lvl4):
    g, _ = lvl4
    b = np.random.default_rng(2).standard_normal(g.n)
    xo, it, rr = orc.gmres(_exported_operator(orc, g, True), b, restart=30, tol=1e-12)
    for precond in (0, 1):
        x, info = g.solve(b, trans=1, rel_tol=1e-12, precond=precond)
        assert info.status == 0 and info.rel_resid <= 1e-12
        r = b - g.matvec(x, trans=1)
        assert np.linalg.norm(r) <= 1.01e-12 * np.linalg.norm(b)
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-8


def test_potential_and_adjoint(orc, lvl4):
    g, cfg = lvl4
    torch = g.torch
    hm = g.hm
    pts = cfg["points"][:256]
    E = orc.potential_matrix(g.V, g.T, pts)
    rng = np.random.default_rng(3)
    a, r = rng.standard_normal(g.n), rng.standard_normal(pts.shape[0])
    pd = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    u = hm.hm_potential(g.tree, pd, torch.from_numpy(a).cuda()).cpu().numpy()
    assert np.abs(u - E @ a).max() <= 1e-13 * (np.abs(E) @ np.abs(a)).max()
    gt = hm.hm_potential(g.tree, pd, torch.from_numpy(r).cuda(), trans=1).cpu().numpy()
    ref = E.T @ r
    assert np.abs(gt - ref).max() <= 1e-13 * (np.abs(E.T) @ np.abs(r)).max()
    # no points: an empty result, and zeros for the adjoint
    e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    z = hm.hm_potential(g.tree, e, torch.empty(0, dtype=torch.float64, device="cuda"), trans=1)
    assert float(z.abs().max()) == 0.0


def misfit_loss(A, tree, f, c, points, target, opts):
    """The differentiation workload's objective: L = mean_k (E alpha - target)_k^2
    with H diag(c) alpha = f, through the library's autograd functions."""
    import torch
    from paper_1806_11558_gb300.autograd import DensitySolve, Potential
    alpha = DensitySolve.apply(A, f, c, opts)
    phi = Potential.apply(tree, points, alpha)
    return torch.mean((phi - target) ** 2)


def _gpu_loss_and_grads(g, cfg, f, c, opts):
    torch = g.torch
    pts = torch.from_numpy(np.ascontiguousarray(cfg["points"])).cuda()
    target = torch.from_numpy(np.ascontiguousarray(_target(cfg))).cuda()
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda().requires_grad_(True)
    cd = torch.from_numpy(np.ascontiguousarray(c)).cuda().requires_grad_(True)
    L = misfit_loss(g.A, g.tree, fd, cd, pts, target, opts)
    L.backward()
    return float(L.detach()), fd.grad.cpu().numpy(), cd.grad.cpu().numpy()


def _target(cfg):
    p = np.asarray(cfg["target_source"])
    return 1.0 / (4.0 * np.pi * np.linalg.norm(cfg["points"] - p[None, :], axis=1))


OPTS = dict(rel_tol=1e-13, restart=128, max_iter=5000, precond=1)


def test_scaled_product_and_solves(orc, lvl4):
    """hm_matvec_scaled and hm_solve_scaled (the column-scaled operator
    H diag(c) of the per-panel coefficients) against the oracle applying the
    exported operator with the scalings written out."""
    g, _ = lvl4
    torch, hm = g.torch, g.hm
    rng = np.random.default_rng(7)
    c = 1.0 + 0.2 * rng.uniform(-1.0, 1.0, g.n)
    l = rng.uniform(0.5, 1.5, g.n)
    x = rng.standard_normal((2, g.n))
    y0 = rng.standard_normal((2, g.n))
    mv, mvt = _exported_operator(orc, g, False), _exported_operator(orc, g, True)
    cd, ld, xd = (torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (c, l, x))
    for trans, op in ((0, mv), (1, mvt)):
        yd = torch.from_numpy(y0.copy()).cuda()
        hm.hm_matvec_scaled(g.A, xd, yd, trans=trans, left=ld, right=cd, alpha=-0.75, beta=0.5)
        torch.cuda.synchronize()
        ref = np.array([-0.75 * l * op(c * x[r]) + 0.5 * y0[r] for r in range(2)])
        assert np.linalg.norm(yd.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
        # identities: no scaling on either side
        yd = torch.empty_like(xd)
        hm.hm_matvec_scaled(g.A, xd, yd, trans=trans)
        torch.cuda.synchronize()
        ref = np.array([op(x[r]) for r in range(2)])
        assert np.linalg.norm(yd.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    b = rng.standard_normal(g.n)
    for trans in (0, 1):
        if trans == 0:
            A_c = lambda v: mv(c * v)
        else:
            A_c = lambda v: c * mvt(v)
        xo, _, _ = orc.gmres(A_c, b, restart=60, tol=1e-13)
        xg = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        info = hm.hm_solve_scaled(g.A, torch.from_numpy(b).cuda(), cd, xg, trans=trans, **OPTS)
        torch.cuda.synchronize()
        assert info.status == 0
        assert np.linalg.norm(xg.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)


def test_misfit_gradients_vs_dense_oracle(orc, lvl4):
    g, cfg = lvl4
    f = orc.load_vector(g.V, g.T, cfg["sources"][0])[0]
    c = 1.0 + 0.1 * np.random.default_rng(4).uniform(-1.0, 1.0, g.n)
    L, gf, gc = _gpu_loss_and_grads(g, cfg, f, c, OPTS)
    A = orc.dense_matrix(g.V, g.T)
    E = orc.potential_matrix(g.V, g.T, cfg["points"])
    Lo, alpha, gfo, gco = orc.misfit_loss_and_gradients(A, E, f, c, _target(cfg))
    # H at eps = 1e-10 is within ~1e-10 of A: gradients within a small multiple of kappa eps
    assert abs(L - Lo) <= 1e-7 * Lo
    assert np.linalg.norm(gf - gfo) <= 1e-6 * np.linalg.norm(gfo)
    assert np.linalg.norm(gc - gco) <= 1e-6 * np.linalg.norm(gco)


def test_misfit_gradients_central_differences_level6(orc):
    """The differentiation workload (level 6, 1,024 points): the autograd
    gradients against central differences (h = 1e-6) on 32 seeded
    directions, 16 in the Dirichlet data and 16 in the panel coefficients."""
    need_gpu()
    cfg = meshgen.config("differentiation")
    g = GpuH(cfg["V"], cfg["T"], leaf=64, eta=1.5, eps=1e-6, kmax=64)
    try:
        torch = g.torch
        f = g.load_vector(cfg["sources"])[0]
        c = np.ones(g.n)
        L0, gf, gc = _gpu_loss_and_grads(g, cfg, f, c, OPTS)
        pts = torch.from_numpy(np.ascontiguousarray(cfg["points"])).cuda()
        target = torch.from_numpy(np.ascontiguousarray(_target(cfg))).cuda()

        def loss(ff, cc):
            with torch.no_grad():
                return float(misfit_loss(g.A, g.tree, torch.from_numpy(ff).cuda(), torch.from_numpy(cc).cuda(),
                                         pts, target, OPTS))

        rng = np.random.default_rng(6)
        h = 1e-6
        worst = 0.0
        for k in range(32):
            # entries of order one relative to the data: every entry moves by ~h
            d = rng.standard_normal(g.n)
            if k < 16:
                df = d * np.abs(f).mean()
                fd = (loss(f + h * df, c) - loss(f - h * df, c)) / (2 * h)
                an = gf @ df
            else:
                fd = (loss(f, c + h * d) - loss(f, c - h * d)) / (2 * h)
                an = gc @ d
            # solver noise: residual 1e-13 times kappa (~1e2 here) over h
            worst = max(worst, abs(fd - an) / abs(an))
            assert abs(fd - an) <= 1e-4 * abs(an) + 1e-9 * L0, (k, fd, an)
        print("worst relative FD deviation over 32 directions: %.2e" % worst)
    finally:
        g.close()
