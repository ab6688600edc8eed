"""Backward pass (mr3_backward): closed forms, invariants, a dense-eigh autograd reference,
and central finite differences of the loss sum(g . lambda) + sum(G o Z)."""
import numpy as np
import pytest

import oracle
import testmats as tm

pytestmark = pytest.mark.gpu


def _fwd(d, e):
    import torch
    import paper_1401_4950_gb300 as mr3
    w, Z, _ = mr3.stemr(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"))
    return w, Z


def _bwd(w, Z, g=None, G=None):
    import torch
    import paper_1401_4950_gb300 as mr3
    gt = None if g is None else torch.tensor(g, device="cuda")
    Gt = None if G is None else torch.tensor(G, device="cuda").t().contiguous().t()
    dd, de = mr3.backward(w, Z, gt, Gt)
    torch.cuda.synchronize()
    return dd.cpu().numpy(), de.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 50, 1000])
def test_eigenvalue_part_closed_forms(cuda, n):
    d, e = tm.random_uniform(n, 11, 12)
    w, Z = _fwd(d, e)
    # sum lambda = trace T  =>  dbar = 1, ebar = 0
    dd, de = _bwd(w, Z, g=np.ones(n))
    assert np.max(np.abs(dd - 1.0)) <= 1e-12 and (n == 1 or np.max(np.abs(de)) <= 1e-12)
    # sum lambda^2 / 2 = ||T||_F^2 / 2  =>  dbar = d, ebar = 2 e
    dd, de = _bwd(w, Z, g=w.cpu().numpy())
    assert np.max(np.abs(dd - d)) <= 1e-12
    if n > 1:
        assert np.max(np.abs(de - 2 * e)) <= 1e-12


def test_vector_part_vanishes_for_G_equal_Z(cuda):
    # dz_i is orthogonal to z_i for unit vectors, so G = Z contributes nothing
    d, e = tm.random_uniform(300, 21, 22)
    w, Z = _fwd(d, e)
    dd, de = _bwd(w, Z, g=None, G=Z.cpu().numpy())
    assert np.max(np.abs(dd)) <= 1e-9 and np.max(np.abs(de)) <= 1e-9


def _loss_grad_dense(d, e, g, G):
    """Reference gradient through torch.linalg.eigh (autograd) on the dense T, CPU FP64,
    with the eigenvector signs of the CUDA solve."""
    import torch
    dt = torch.tensor(d, requires_grad=True)
    et = torch.tensor(e, requires_grad=True)
    T = torch.diag(dt) + torch.diag(et, 1) + torch.diag(et, -1)
    lam, V = torch.linalg.eigh(T)
    return dt, et, lam, V


@pytest.mark.parametrize("n", [20, 128, 400])
def test_matches_dense_eigh_autograd(cuda, n):
    import torch
    d, e = tm.random_uniform(n, 31, 32)
    g = tm.normal(33, n)
    G = tm.normal(34, n * n).reshape(n, n)
    w, Z = _fwd(d, e)
    dd, de = _bwd(w, Z, g=g, G=G)
    dt, et, lam, V = _loss_grad_dense(d, e, g, G)
    Zc = Z.cpu().numpy()
    s = np.sign(np.einsum("ij,ij->j", V.detach().numpy(), Zc))
    loss = (torch.tensor(g) * lam).sum() + (torch.tensor(G) * (V * torch.tensor(s))).sum()
    loss.backward()
    scale = max(np.abs(dt.grad.numpy()).max(), 1.0)
    assert np.max(np.abs(dd - dt.grad.numpy())) <= 1e-8 * scale
    assert np.max(np.abs(de - et.grad.numpy())) <= 1e-8 * scale


def _separated(n, seed):
    """Tridiagonal with well-separated eigenvalues (8 (i + U(-0.1, 0.1)) / n on the diagonal,
    2.4 U(-1, 1) / n off it, so ||T|| ~ 8 and gaps ~ 6/n): central differences of
    eigenvalues have truncation error ~(h/gap)^2 and rounding noise ~eps ||T|| / h, while
    random tridiagonals have near-crossings (Poisson-like level statistics)."""
    d = 8.0 * (np.arange(n, dtype=np.float64) + 0.1 * tm.uniform(seed, n)) / n
    e = 2.4 * tm.uniform(seed + 1, n - 1) / n
    return d, e


@pytest.mark.parametrize("n", [64, 512])
def test_central_finite_differences_eigenvalue_part(cuda, n):
    # eigenvalues are determined to ~n eps ||T||, so central differences at h = 1e-6 of
    # sum(g . lambda) resolve the gradient to ~1e-8 relative when the gaps are O(1)
    d, e = _separated(n, 41)
    g = tm.normal(43, n)
    w, Z = _fwd(d, e)
    assert np.diff(w.cpu().numpy()).min() > 1.0 / n
    dd, de = _bwd(w, Z, g=g)

    def loss(dv, ev):
        wv, _ = _fwd(dv, ev)
        return float(g @ wv.cpu().numpy())

    h = 1e-6
    for k in range(3):
        # unit direction, so that the perturbation h V of T has norm ~h
        vd = tm.normal(500 + 2 * k, n)
        ve = tm.normal(501 + 2 * k, n - 1)
        nv = np.sqrt(vd @ vd + 2 * ve @ ve)
        vd, ve = vd / nv, ve / nv
        fd = (loss(d + h * vd, e + h * ve) - loss(d - h * vd, e - h * ve)) / (2 * h)
        an = float(dd @ vd + de @ ve)
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def _ld_jacobi(d, e):
    """Eigen-decomposition of the dense T by cyclic Jacobi in numpy longdouble (80-bit
    extended on x86, 128-bit on aarch64): rounding noise far below what a central
    difference at h = 1e-6 can see.  Returns ascending eigenvalues and column vectors."""
    n = len(d)
    A = np.zeros((n, n), dtype=np.longdouble)
    A[np.arange(n), np.arange(n)] = d
    A[np.arange(n - 1), np.arange(1, n)] = e
    A[np.arange(1, n), np.arange(n - 1)] = e
    V = np.eye(n, dtype=np.longdouble)
    one = np.longdouble(1)
    for _ in range(60):
        off = np.sqrt(np.sum(A * A) - np.sum(np.diag(A) ** 2))
        if off < np.finfo(np.longdouble).eps * 1e-2:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0:
                    continue
                theta = (A[q, q] - A[p, p]) / (2 * apq)
                t = (one if theta >= 0 else -one) / (abs(theta) + np.sqrt(one + theta * theta))
                c = one / np.sqrt(one + t * t)
                sn = t * c
                Ap, Aq = A[:, p].copy(), A[:, q].copy()
                A[:, p], A[:, q] = c * Ap - sn * Aq, sn * Ap + c * Aq
                Ap, Aq = A[p, :].copy(), A[q, :].copy()
                A[p, :], A[q, :] = c * Ap - sn * Aq, sn * Ap + c * Aq
                Vp, Vq = V[:, p].copy(), V[:, q].copy()
                V[:, p], V[:, q] = c * Vp - sn * Vq, sn * Vp + c * Vq
    w = np.diag(A).copy()
    o = np.argsort(w)
    return w[o], V[:, o]


def test_central_finite_differences_full_loss(cuda):
    # full loss sum(g . lambda) + sum(G o Z): central differences (h = 1e-6) of an
    # extended-precision forward against the backward of the CUDA forward, 1e-6 relative
    n = 16
    d, e = tm.random_uniform(n, 51, 52)
    g = tm.normal(53, n)
    G = tm.normal(54, n * n).reshape(n, n)
    w, Z = _fwd(d, e)
    Z0 = Z.cpu().numpy()
    dd, de = _bwd(w, Z, g=g, G=G)
    h = 1e-6
    vd = tm.normal(55, n)
    ve = tm.normal(56, n - 1)

    def loss(sign):
        dv = d.astype(np.longdouble) + sign * np.longdouble(h) * vd.astype(np.longdouble)
        ev = e.astype(np.longdouble) + sign * np.longdouble(h) * ve.astype(np.longdouble)
        wv, V = _ld_jacobi(dv, ev)
        s = np.sign(np.einsum("ij,ij->j", V.astype(np.float64), Z0))
        return np.sum(g.astype(np.longdouble) * wv) + np.sum(G.astype(np.longdouble) * V * s)

    fd = float((loss(1) - loss(-1)) / (2 * np.longdouble(h)))
    an = float(dd @ vd + de @ ve)
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_central_finite_differences_gpu_forward_full_loss(cuda):
    # with the FP64 forward itself the eigenvector part of the loss carries O(n eps / gap)
    # noise, amplified 1/h by the difference quotient; the agreement is bounded by that
    import torch
    n = 64
    d, e = tm.random_uniform(n, 41, 42)
    g = tm.normal(43, n)
    G = tm.normal(44, n * n).reshape(n, n)
    w, Z = _fwd(d, e)
    Z0 = Z.cpu().numpy()
    dd, de = _bwd(w, Z, g=g, G=G)

    def loss(dv, ev):
        wv, Zv = _fwd(dv, ev)
        Zv = Zv.cpu().numpy()
        Zv = Zv * np.sign(np.einsum("ij,ij->j", Z0, Zv))[None, :]
        return float(g @ wv.cpu().numpy() + (G * Zv).sum())

    h = 1e-6
    vd = tm.normal(500, n)
    ve = tm.normal(501, n - 1)
    fd = (loss(d + h * vd, e + h * ve) - loss(d - h * vd, e - h * ve)) / (2 * h)
    an = float(dd @ vd + de @ ve)
    assert abs(fd - an) <= 1e-3 * abs(an), (fd, an)


def test_fd_against_oracle_forward(cuda):
    # the backward pinned to finite differences of the CPU oracle's eigen-decomposition
    import torch
    n = 40
    d, e = tm.random_uniform(n, 61, 62)
    g = tm.normal(63, n)
    G = tm.normal(64, n * n).reshape(n, n)
    w, Z = _fwd(d, e)
    Z0 = Z.cpu().numpy()
    dd, de = _bwd(w, Z, g=g, G=G)

    def loss(dv, ev):
        wv = oracle.eigvals(dv, ev)
        Zv = oracle.eigvecs(dv, ev, wv)
        Zv = Zv * np.sign(np.einsum("ij,ij->j", Z0, Zv))[None, :]
        return float(g @ wv + (G * Zv).sum())

    h = 1e-6
    vd = tm.normal(70, n)
    ve = tm.normal(71, n - 1)
    fd = (loss(d + h * vd, e + h * ve) - loss(d - h * vd, e - h * ve)) / (2 * h)
    an = float(dd @ vd + de @ ve)
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_autograd_function(cuda):
    import torch
    import paper_1401_4950_gb300 as mr3
    n = 100
    d, e = tm.random_uniform(n, 81, 82)
    dt = torch.tensor(d, device="cuda", requires_grad=True)
    et = torch.tensor(e, device="cuda", requires_grad=True)
    w, Z = mr3.eigh_tridiagonal(dt, et)
    (w.sum()).backward()
    assert torch.allclose(dt.grad, torch.ones_like(dt), atol=1e-12)
    assert torch.max(torch.abs(et.grad)).item() <= 1e-12


def _vector_part_fp64(w, Z, G):
    """dbar, ebar of the vector part in plain binary64 on the CPU (the formula written out:
    B = F o (Z^T G), Y = Z B, dbar_j = sum_k Y_jk Z_jk, ebar_j = sum_k Y_jk Z_j+1,k +
    Y_j+1,k Z_jk), with the regularised F and delta = n eps ||T|| of the library."""
    n = len(w)
    delta = n * 2.0 ** -53 * max(abs(w[0]), abs(w[-1]))
    D = w[None, :] - w[:, None]
    F = D / (D * D + delta * delta)
    np.fill_diagonal(F, 0.0)
    Y = Z @ (F * (Z.T @ G))
    dd = np.einsum("jk,jk->j", Y, Z)
    de = np.einsum("jk,jk->j", Y[:-1], Z[1:]) + np.einsum("jk,jk->j", Y[1:], Z[:-1])
    return dd, de


@pytest.mark.parametrize("n,kind", [(256, "random"), (700, "random"), (1500, "one_two_one"),
                                    (4500, "random")])
def test_split_product_backward_matches_fp64(cuda, n, kind):
    # the vector part through the bf16 slice products (n >= 256; two contraction chunks
    # at n = 4500) against the same formula in binary64
    d, e = tm.make(kind, n, seed=91)
    G = tm.normal(92, n * n).reshape(n, n)
    w, Z = _fwd(d, e)
    dd, de = _bwd(w, Z, g=None, G=G)
    wc, Zc = w.cpu().numpy(), Z.cpu().numpy()
    rd, re_ = _vector_part_fp64(wc, Zc, G)
    scale = max(np.abs(rd).max(), np.abs(re_).max())
    assert np.max(np.abs(dd - rd)) <= 1e-11 * scale, np.max(np.abs(dd - rd)) / scale
    assert np.max(np.abs(de - re_)) <= 1e-11 * scale, np.max(np.abs(de - re_)) / scale


def test_split_product_wide_dynamic_range(cuda):
    # columns of G spanning 2^-300 .. 2^300 and entries 2^20 apart inside a column: the
    # power-of-two scaling per line keeps the slices in range (no overflow, no flush to 0)
    n = 512
    d, e = tm.make("random", n, seed=93)
    G = tm.normal(94, n * n).reshape(n, n)
    G *= np.exp2(np.linspace(-300, 300, n))[None, :]
    G[::7] *= 2.0 ** -20
    w, Z = _fwd(d, e)
    dd, de = _bwd(w, Z, g=None, G=G)
    rd, re_ = _vector_part_fp64(w.cpu().numpy(), Z.cpu().numpy(), G)
    scale = max(np.abs(rd).max(), np.abs(re_).max())
    assert np.all(np.isfinite(dd)) and np.all(np.isfinite(de))
    assert np.max(np.abs(dd - rd)) <= 1e-11 * scale
    assert np.max(np.abs(de - re_)) <= 1e-11 * scale


def test_backward_workload_eigenvalue_part_fd(cuda):
    # the backward workload's matrix (n = 4096, uniform(-1, 1), seeds 501, 502), loss
    # sum(g . lambda) with g ~ N(0, 1) (seed 503): central differences at h = 1e-6 along two
    # random unit directions agree to 1e-6 of the gradient's norm (the difference quotient's
    # own noise is ~sqrt(n) eps ||T|| / h ~ 1e-7 absolute, so a direction with a small
    # derivative cannot be held to 1e-6 of itself).  Off-diagonals near zero almost split
    # such a matrix, so some eigenvalue pairs sit at avoided crossings with gaps far below
    # h, across which a single eigenvalue is not smooth at that step; the sum over such a
    # group is, so g is made constant within groups closer than 1e-4.
    n = 4096
    d, e = tm.random_uniform(n, 501, 502)
    g = tm.normal(503, n)
    w, Z = _fwd(d, e)
    wc = w.cpu().numpy()
    for i in range(1, n):
        if wc[i] - wc[i - 1] < 1e-4:
            g[i] = g[i - 1]
    dd, de = _bwd(w, Z, g=g)
    gnorm = np.sqrt(dd @ dd + 0.5 * de @ de)  # dual norm of the unit directions below

    def loss(dv, ev):
        wv, _ = _fwd(dv, ev)
        return float(g @ wv.cpu().numpy())

    h = 1e-6
    for k in range(2):
        vd = tm.normal(505 + 2 * k, n)
        ve = tm.normal(506 + 2 * k, n - 1)
        nv = np.sqrt(vd @ vd + 2 * ve @ ve)
        vd, ve = vd / nv, ve / nv
        fd = (loss(d + h * vd, e + h * ve) - loss(d - h * vd, e - h * ve)) / (2 * h)
        an = float(dd @ vd + de @ ve)
        assert abs(fd - an) <= 1e-6 * gnorm, (fd, an, gnorm)


def test_backward_full_loss_fd_n4096_double_double_forward(cuda):
    # loss sum(g . lambda) + sum(G o Z) at n = 4096 on a matrix with gaps ~8/n, the forward
    # through the double-double tree (eigenvectors accurate far below what h = 1e-6 can
    # see): central differences along a random unit direction against the backward
    import torch
    import paper_1401_4950_gb300 as mr3
    n = 4096
    d, e = _separated(n, 61)
    g = tm.normal(62, n)
    G = tm.normal(63, n * n).reshape(n, n)
    opts = mr3.make_opts(prec=mr3.DD)

    def fwd(dv, ev):
        w, Z, _ = mr3.stemr(torch.tensor(dv, device="cuda"), torch.tensor(ev, device="cuda"),
                            opts=opts)
        return w, Z

    w0, Z0 = fwd(d, e)
    dd, de = _bwd(w0, Z0, g=g, G=G)
    Z0c = Z0.cpu().numpy()
    Gt = torch.tensor(G, device="cuda")

    def loss(dv, ev):
        w, Z = fwd(dv, ev)
        s = torch.sign(torch.einsum("ij,ij->j", Z, torch.tensor(Z0c, device="cuda")))
        return float(torch.tensor(g, device="cuda") @ w + torch.sum(Gt * (Z * s[None, :])))

    h = 1e-6
    vd = tm.normal(64, n)
    ve = tm.normal(65, n - 1)
    nv = np.sqrt(vd @ vd + 2 * ve @ ve)
    vd, ve = vd / nv, ve / nv
    fd = (loss(d + h * vd, e + h * ve) - loss(d - h * vd, e - h * ve)) / (2 * h)
    an = float(dd @ vd + de @ ve)
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
