"""Pins of the oracle's Gram-Schmidt, projection, reduced poles and IRKA
(Algorithm 2 with N_j = 0; reuse schedule of Algorithm 4) against the
interpolation theory of Sec. II, closed forms and LAPACK."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import irka, operator as op


def test_cgs2_orthogonality_span_and_factorisation():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((500, 8))
    X[:, 5] = X[:, 4] + 1e-7 * rng.standard_normal(500)     # nearly dependent
    V, R = irka.cgs2(X)
    assert np.linalg.norm(V.T @ V - np.eye(8)) <= 1e-13
    assert np.linalg.norm(X - V @ V.T @ X) <= 1e-10 * np.linalg.norm(X)
    np.testing.assert_allclose(V @ R, X, atol=1e-12)
    assert np.allclose(R, np.triu(R))


def test_reduced_poles_known_spectra():
    # diagonal pencil
    a = np.array([-1.0, -2.0, -3.5])
    e = np.array([2.0, 1.0, 0.5])
    lam = np.sort_complex(irka.reduced_poles(np.diag(a), np.diag(e)))
    np.testing.assert_allclose(lam, np.sort_complex(a / e))
    # companion matrix of (x+1)(x+2)(x^2+2x+5) -> roots -1, -2, -1 +- 2i
    c = np.poly([-1, -2, -1 + 2j, -1 - 2j]).real
    Cmp = np.zeros((4, 4))
    Cmp[0, :] = -c[1:]
    Cmp[1:, :-1] = np.eye(3)
    lam = irka.reduced_poles(Cmp, np.eye(4))
    want = np.array([-1, -2, -1 + 2j, -1 - 2j])
    for w in want:
        assert np.min(np.abs(lam - w)) < 1e-10


def test_mirror_sort_and_pairing():
    lam = np.array([-3 + 1j, -1.0, -3 - 1j, 2.0 + 0.5j, 2.0 - 0.5j])
    s = irka.mirror_shifts(lam)
    # -lambda for stable poles; reflection for the unstable pair; pairs adjacent, +Im first
    assert s[0] == 1.0
    assert s[1] == 2.0 + 0.5j and s[2] == 2.0 - 0.5j
    assert s[3] == 3.0 + 1j and s[4] == 3.0 - 1j
    sol = irka.solve_shifts_of(s)
    assert list(sol) == [1.0, 2.0 + 0.5j, 3.0 + 1j]


def _dense_run(wl, iters, mode="reuse"):
    return irka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=iters, solver="dense",
                     mode=mode, hermite=True)


@pytest.mark.parametrize("which", ["sym", "nonsym"])
def test_hermite_interpolation_every_iteration(which):
    """Petrov-Galerkin with V, W from the shifted solves interpolates H and
    H' at every shift, at every iteration (Sec. II)."""
    wl = W.config0(N=9) if which == "sym" else W.config1(N=5)
    res = _dense_run(wl, 4)
    for h in res.hermite:
        np.testing.assert_allclose(h["Hr"], h["H"], rtol=1e-9)
        np.testing.assert_allclose(h["dHr"], h["dH"], rtol=1e-8)


def test_full_order_reduction_reproduces_H():
    """r = n: V and W span R^n, so H_r == H at any frequency."""
    wl = W.random_sparse_system(6, 0.5, seed=9, e_kind="diag")
    shifts = np.array([1.0, 2.0 + 1.0j, 2.0 - 1.0j, 5.0, 8.0, 13.0], dtype=complex)
    res = irka.irka(wl.A, wl.E, wl.B, wl.C, shifts, iters=1, solver="dense")
    w = np.logspace(-1, 2, 7) * 1j
    H = op.transfer_function(wl.A, wl.E, wl.B, wl.C, w)
    Hr = op.transfer_function_reduced(res.Ar, res.Er, res.Br, res.Cr, w)
    np.testing.assert_allclose(Hr, H, rtol=1e-10)


def test_irka_fixed_point_is_mirrored_reduced_poles():
    """Converged IRKA: sigma_i = -lambda_i(A_r, E_r)."""
    rng = np.random.default_rng(4)
    n = 40
    a = -np.sort(rng.uniform(1, 100, n))
    A = sp.diags(a, format="csr")
    B = rng.standard_normal((n, 1))
    C = rng.standard_normal((n, 1))
    res = irka.irka(A, None, B, C, np.array([2.0, 20.0, 60.0], dtype=complex), iters=60, solver="dense")
    s_last, s_prev = res.shifts_history[-1], res.shifts_history[-2]
    assert np.max(np.abs(s_last - s_prev) / np.abs(s_last)) < 1e-9
    lam = irka.reduced_poles(res.Ar, res.Er)
    np.testing.assert_allclose(np.sort_complex(-lam), np.sort_complex(s_prev), rtol=1e-8)


def test_iterative_irka_matches_dense_irka():
    """BiCGSTAB with reused SPAI (Algorithm 4) to 1e-8 reproduces the exact
    (dense LU) IRKA's H_r to 1e-6 on log-spaced frequencies."""
    wl = W.config1(N=8)
    rd = _dense_run(wl, 3)
    ri = irka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=3, solver="bicgstab")
    w = 1j * np.logspace(0, 5, 200)
    Hd = op.transfer_function_reduced(rd.Ar, rd.Er, rd.Br, rd.Cr, w)[:, 0, 0]
    Hi = op.transfer_function_reduced(ri.Ar, ri.Er, ri.Br, ri.Cr, w)[:, 0, 0]
    H = op.transfer_function(wl.A, wl.E, wl.B, wl.C, w)[:, 0, 0]
    assert np.max(np.abs(Hi - Hd) / np.abs(H)) <= 1e-6


def test_reuse_schedule_follows_algorithm4():
    wl = W.config1(N=5)
    res = irka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=3, solver="dense")
    prim = [b for b in res.builds[: len(res.builds) // 2]]
    # z = 1: full SPAI for i = 1, horizontal for i > 1
    assert prim[0] == (1, 1, "spai")
    assert all(k == "horizontal" for (z, i, k) in prim if i > 1)
    assert [k for (z, i, k) in prim if i == 1] == ["spai", "vertical", "vertical"]


def test_reuse_vs_fresh_vs_none_same_rom():
    """The preconditioner changes iteration counts, never the solution:
    reuse, fresh-SPAI and unpreconditioned IRKA give the same H_r."""
    wl = W.config0(N=12)
    w = 1j * np.logspace(0, 5, 50)
    Hs = []
    for mode in ("reuse", "fresh", "none"):
        r = irka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=2, mode=mode)
        Hs.append(op.transfer_function_reduced(r.Ar, r.Er, r.Br, r.Cr, w)[:, 0, 0])
    H = op.transfer_function(wl.A, wl.E, wl.B, wl.C, w)[:, 0, 0]
    for Hx in Hs[1:]:
        assert np.max(np.abs(Hx - Hs[0]) / np.abs(H)) <= 1e-6
