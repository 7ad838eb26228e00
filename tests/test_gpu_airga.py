"""GPU parity of the second-order reduction (mor_airga_step, AIRGA iteration
of Algorithm 1 with the reuse schedule) against the oracle:

  * expansion points of every iteration within 20 x the oracle's own
    movement between solve tolerances 1e-8 and 1e-10 (at least 1e-6);
  * the 2r eigenvalues of the reduced quadratic eigenproblem of the GPU's
    M_r, D_r, K_r match the oracle's within 20 x the oracle's own movement of
    those eigenvalues between the two tolerances (at least 1e-6): the
    high-frequency ones are the least determined by a reduced model that
    interpolates at low-frequency points;
  * moment matching H_r(s_i) = H(s_i) at the solved points to 1e-6 with the
    exact H (these lightly damped systems make H_r on a frequency grid an
    ill-conditioned measure: a pole moved by 1e-8 moves H_r near its
    resonance by ~1e-8 / damping ratio);
  * mor_eval_tf2 evaluates the reduced transfer function of a given ROM to
    1e-10 of the oracle's dense evaluation.
"""
import numpy as np
import pytest

import paper_2003_12759_gb300 as mor
import workloads as W
from oracle import airga

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    mor.load_library()
    hh = mor.mor_create(0)
    yield hh
    mor.mor_destroy(hh)


def _set(h, wl):
    mor.mor_set_system_2nd(h, wl.K, wl.M_diag, wl.alpha, wl.beta, wl.F, wl.C)


POINTS = np.array([0.2 + 0.1j, 0.2 - 0.1j, 1.0])


def _H(wl, s):
    return airga.transfer_function_2nd(wl.K, wl.M_diag, wl.alpha, wl.beta, wl.F, wl.C, [s])[0]


@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
@pytest.mark.parametrize("dims", [(9, 8, 7, 3), (6, 7, 5, 4)])
def test_airga_matches_oracle(h, precision, dims):
    nx, ny, nz, m = dims
    wl = W.stencil27_second_order(nx=nx, ny=ny, nz=nz, m=m)
    iters = 3
    a, sa = airga.airga(wl.K, wl.M_diag, wl.alpha, wl.beta, wl.F, wl.C, POINTS, iters=iters, tol=1e-8)
    b, sb = airga.airga(wl.K, wl.M_diag, wl.alpha, wl.beta, wl.F, wl.C, POINTS, iters=iters, tol=1e-10)
    move = max(np.max(np.abs(x - y) / np.abs(y)) for x, y in zip(a.shifts_history[1:], b.shifts_history[1:]))
    bar = max(1e-6, 20.0 * move)
    emove = 0.0
    for (_, ra), (_, rb) in zip(sa, sb):
        la, lb = airga.qep_eigenvalues(*ra[:3]), airga.qep_eigenvalues(*rb[:3])
        emove = max(emove, max(np.min(np.abs(la - z)) / abs(z) for z in lb))
    ebar = max(1e-6, 20.0 * emove)
    _set(h, wl)
    p = POINTS.copy()
    opts = mor.mor_default_opts(precision=precision)
    for z in range(iters):
        solved = [x for x in airga.sort_shifts(p) if x.imag >= 0]
        p, rom, st = mor.mor_airga_step(h, p, opts)
        assert st["max_relres"] <= 1.001e-8
        assert rom.r == m * len(POINTS)
        so = a.shifts_history[z + 1]
        assert np.max(np.abs(p - so) / np.abs(so)) <= bar, (z, p, so, bar)
        Mr, Dr, Kr, Fr, Cr = rom.arrays()
        lg = airga.qep_eigenvalues(Mr, Dr, Kr)
        lo = airga.qep_eigenvalues(*sa[z][1][:3])
        for zz in lo:
            assert np.min(np.abs(lg - zz)) <= ebar * abs(zz), (zz, ebar)
        for s in solved:
            H = _H(wl, s)
            Hr = airga.transfer_function_2nd_reduced(Mr, Dr, Kr, Fr, Cr, [s])[0]
            assert np.linalg.norm(Hr - H) <= 1e-6 * np.linalg.norm(H)


def test_eval_tf2_matches_dense_evaluation(h):
    wl = W.stencil27_second_order(nx=6, ny=5, nz=4, m=2)
    _set(h, wl)
    p, rom, _ = mor.mor_airga_step(h, POINTS, mor.mor_default_opts(precision=mor.MOR_FP64))
    w = np.logspace(-2, 1, 300)
    Hg = mor.mor_eval_tf2(h, rom, w)
    Ho = airga.transfer_function_2nd_reduced(*rom.arrays(), 1j * w)
    assert np.max(np.abs(Hg - Ho)) <= 1e-10 * np.max(np.abs(Ho))


def test_airga_argument_errors(h):
    wl = W.stencil27_second_order(nx=5, ny=4, nz=4, m=4)
    _set(h, wl)
    with pytest.raises(RuntimeError):                 # r = 4 * 9 > 32
        mor.mor_airga_step(h, np.linspace(0.1, 1.0, 9), mor.mor_default_opts())
    with pytest.raises(RuntimeError):                 # not closed under conjugation
        mor.mor_airga_step(h, np.array([0.2 + 0.1j, 1.0]), mor.mor_default_opts())
    first = W.convdiff3d_siso(N=5)
    mor.mor_set_system(h, first.A, first.B, first.C, E_diag=first.E)
    with pytest.raises(RuntimeError):
        mor.mor_airga_step(h, POINTS, mor.mor_default_opts())


def _derivs2(wl, Mm, D, K, F, C, s, order):
    """H, H', H'' of C^T (s^2 M + s D + K)^{-1} F (dense closed forms:
    H' = -C^T A^{-1} A' A^{-1} F, H'' = C^T (2 A^{-1} A' A^{-1} A' A^{-1} -
    A^{-1} A'' A^{-1}) F, A' = 2 s M + D, A'' = 2 M)."""
    A = s * s * Mm + s * D + K
    A1 = 2 * s * Mm + D
    X0 = np.linalg.solve(A, F.astype(complex))
    out = [C.T @ X0]
    if order >= 1:
        X1 = np.linalg.solve(A, A1 @ X0)
        out.append(-(C.T @ X1))
    if order >= 2:
        X2 = np.linalg.solve(A, A1 @ X1)
        out.append(C.T @ (2 * X2 - np.linalg.solve(A, 2 * Mm @ X0)))
    return out


@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
@pytest.mark.parametrize("J", [2, 3])
def test_airga_moment_loop_matches_oracle(h, J, precision):
    """The inner moment loop on the GPU (J blocks X^(j) = -A(s)^{-1} M V_j per
    point, same chain): every iteration's ROM has r = m J l and matches H and
    its first J - 1 derivatives at every solved point and its conjugate
    (1e-6; the oracle reaches <= 1e-9 with 1e-8 solves); the first
    iteration's reduced QEP eigenvalues and the next points agree with the
    oracle's within 20 x its own movement between solve tolerances 1e-8 and
    1e-10 (the moment blocks of a point are nearly dependent, which makes
    the points sensitive: 1.5e-4 to 1.8e-3 there)."""
    wl = W.stencil27_second_order(nx=6, ny=5, nz=4, m=2)
    a, sa = airga.airga(wl.K, wl.M_diag, wl.alpha, wl.beta, wl.F, wl.C, POINTS, iters=1, tol=1e-8, moments=J)
    b, sb = airga.airga(wl.K, wl.M_diag, wl.alpha, wl.beta, wl.F, wl.C, POINTS, iters=1, tol=1e-10, moments=J)
    bar = max(1e-6, 20.0 * np.max(np.abs(a.shifts_history[1] - b.shifts_history[1]) / np.abs(b.shifts_history[1])))
    la, lb = airga.qep_eigenvalues(*sa[0][1][:3]), airga.qep_eigenvalues(*sb[0][1][:3])
    ebar = max(1e-6, 20.0 * max(np.min(np.abs(la - z)) / abs(z) for z in lb))
    Mm = np.diag(wl.M_diag)
    K = wl.K.toarray()
    D = wl.alpha * Mm + wl.beta * K
    _set(h, wl)
    p = POINTS.copy()
    opts = mor.mor_default_opts(precision=precision, moments=J)
    for z in range(2):
        solved = [x for x in airga.sort_shifts(p) if x.imag >= 0]
        p, rom, st = mor.mor_airga_step(h, p, opts)
        assert st["max_relres"] <= 1.001e-8
        assert rom.r == 2 * J * len(POINTS) and st["nsolve"] == 2 * J * len(solved)
        Mr, Dr, Kr, Fr, Cr = rom.arrays()
        for s in solved + [np.conj(x) for x in solved if x.imag != 0]:
            full = _derivs2(wl, Mm, D, K, wl.F, wl.C, s, J - 1)
            red = _derivs2(wl, Mr, Dr, Kr, Fr, Cr, s, J - 1)
            for k, (x, y) in enumerate(zip(full, red)):
                assert np.linalg.norm(y - x) <= 1e-6 * np.linalg.norm(x), (z, s, k)
        if z == 0:
            assert np.max(np.abs(p - a.shifts_history[1]) / np.abs(a.shifts_history[1])) <= bar
            lg = airga.qep_eigenvalues(Mr, Dr, Kr)
            for zz in la:
                assert np.min(np.abs(lg - zz)) <= ebar * abs(zz), (zz, ebar)


def test_airga_moments_argument_errors(h):
    wl = W.stencil27_second_order(nx=5, ny=4, nz=4, m=4)
    _set(h, wl)
    with pytest.raises(RuntimeError):                 # r = 4 * 3 * 3 > 32
        mor.mor_airga_step(h, POINTS, mor.mor_default_opts(moments=3))
    with pytest.raises(RuntimeError):
        mor.mor_airga_step(h, POINTS, mor.mor_default_opts(moments=0))
