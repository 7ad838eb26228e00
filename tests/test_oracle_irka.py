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
    wl = W.laplace2d_siso(N=9) if which == "sym" else W.convdiff3d_siso(N=5)
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
    wl = W.convdiff3d_siso(N=8)
    rd = _dense_run(wl, 3)
    ri = irka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=3, solver="bicgstab")
    w = 1j * np.logspace(0, 5, 200)
    Hd = op.transfer_function_reduced(rd.Ar, rd.Er, rd.Br, rd.Cr, w)[:, 0, 0]
    Hi = op.transfer_function_reduced(ri.Ar, ri.Er, ri.Br, ri.Cr, w)[:, 0, 0]
    H = op.transfer_function(wl.A, wl.E, wl.B, wl.C, w)[:, 0, 0]
    assert np.max(np.abs(Hi - Hd) / np.abs(H)) <= 1e-6


def test_reuse_schedule_follows_algorithm4():
    wl = W.convdiff3d_siso(N=5)
    res = irka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=3, solver="dense")
    prim = [b for b in res.builds[: len(res.builds) // 2]]
    # z = 1: full SPAI for i = 1, horizontal for i > 1
    assert prim[0] == (1, 1, "spai")
    assert all(k == "horizontal" for (z, i, k) in prim if i > 1)
    assert [k for (z, i, k) in prim if i == 1] == ["spai", "vertical", "vertical"]


def test_first_approach_chains_and_full_pattern_inverse():
    """Table II's first approach along the shifts: every shift i > 1 gets the
    vertical chain plus one factor Q_i fitted from A_1 (min ||A_1 - A_i Q||_F).
    With a full pattern Q_i = A_i^{-1} A_1 and P_1 = A_1^{-1}, so every chain
    is exactly A_i^{-1}: A_i Q_i P_1 = A_1 P_1 = I (Table II, first column)."""
    wl = W.convdiff3d_siso(N=3)                      # n = 27
    n = wl.A.shape[0]
    s = irka.ReuseSchedule(wl.A, wl.E, transpose=False, mode="first")
    s.S = sp.csr_matrix(np.ones((n, n)))             # full pattern
    shifts = np.array([20.0 + 5.0j, 35.0 + 2.0j, 60.0, 90.0 + 30.0j])
    ch = s.chains(1, shifts)
    assert [len(c) for c in ch] == [1, 2, 2, 2]
    assert [k for (_, _, k) in s.builds] == ["spai", "first", "first", "first"]
    for c, x in zip(ch, shifts):
        M = op.A_sigma(wl.A, wl.E, x).toarray()
        P = np.eye(n, dtype=complex)
        for F in c:
            P = F.toarray() @ P
        assert np.linalg.norm(M @ P - np.eye(n)) <= 1e-9
    ch2 = s.chains(2, shifts * 1.01)                  # second iteration: vertical factor + Q_i
    assert [len(c) for c in ch2] == [2, 3, 3, 3]
    assert all(c[:2] == ch2[0] for c in ch2[1:])


def test_auto_policy_reads_the_frobenius_ratios():
    """The reuse decision (reading of the paper's ratio discussion): close
    shifts (change ratio far below 1 and below ||I - A||_F / ||I||_F) reuse,
    a jump whose change ratio exceeds 1 builds a fresh SPAI, which then
    starts the horizontal chain again; the decision agrees with ratios
    recomputed by brute force on the dense matrices."""
    wl = W.laplace2d_siso(N=8)
    n = wl.A.shape[0]
    s = irka.ReuseSchedule(wl.A, wl.E, transpose=False, mode="auto")
    shifts = np.array([100.0, 110.0, 5000.0, 5100.0])
    ch = s.chains(1, shifts)
    kinds = [k for (_, _, k) in s.builds]
    assert kinds == ["spai", "horizontal", "spai", "horizontal"]
    assert [len(c) for c in ch] == [1, 2, 1, 2]
    for a, b, want in ((100.0, 110.0, True), (110.0, 5000.0, False), (5000.0, 5100.0, True)):
        Ma = op.A_sigma(wl.A, wl.E, a).toarray()
        Mb = op.A_sigma(wl.A, wl.E, b).toarray()
        std = np.linalg.norm(np.eye(n) - Mb) / np.sqrt(n)
        change = np.linalg.norm(Ma - Mb) / np.linalg.norm(Ma)
        assert (change < min(1.0, std)) == want == s.reuse_ok(a, b)
    s.chains(2, shifts * 1.02)                        # small vertical move: reused
    assert s.builds[4] == (2, 1, "vertical")
    s.chains(3, shifts * 40.0)                        # large vertical move: rebuilt
    assert s.builds[8] == (3, 1, "spai")


def test_reuse_vs_fresh_vs_none_same_rom():
    """The preconditioner changes iteration counts, never the solution:
    reuse, first-approach, ratio-policy, fresh-SPAI and unpreconditioned
    IRKA give the same H_r."""
    wl = W.laplace2d_siso(N=12)
    w = 1j * np.logspace(0, 5, 50)
    Hs = []
    for mode in ("reuse", "first", "auto", "fresh", "none"):
        r = irka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=2, mode=mode)
        Hs.append(op.transfer_function_reduced(r.Ar, r.Er, r.Br, r.Cr, w)[:, 0, 0])
    H = op.transfer_function(wl.A, wl.E, wl.B, wl.C, w)[:, 0, 0]
    for Hx in Hs[1:]:
        assert np.max(np.abs(Hx - Hs[0]) / np.abs(H)) <= 1e-6


# ----------------------------------------------------------------------------
# tangential (MIMO) IRKA
# ----------------------------------------------------------------------------
def _mimo(n=50, m=3, q=2, seed=31, e_kind="diag"):
    return W.random_sparse_system(n, 0.08, seed=seed, e_kind=e_kind, m=m, q=q)


def _H_and_dH(wl, s):
    """H(s) = C^T K^{-1} B and H'(s) = -C^T K^{-1} E K^{-1} B, K = sE - A (dense)."""
    K = op.A_sigma(wl.A, wl.E, s).toarray()
    Em = op.E_matrix(wl.E, wl.A.shape[0])
    Em = Em.toarray() if sp.issparse(Em) else Em
    X = np.linalg.solve(K, wl.B.astype(complex))
    return wl.C.T @ X, -(wl.C.T @ np.linalg.solve(K, Em @ X))


def _Hr_and_dHr(rom, s):
    Ar, Er, Br, Cr = rom
    K = s * Er - Ar
    X = np.linalg.solve(K, Br.astype(complex))
    return Cr.T @ X, -(Cr.T @ np.linalg.solve(K, Er @ X))


@pytest.mark.parametrize("e_kind", ["identity", "diag", "csr"])
def test_tangential_bitangential_hermite_every_iteration(e_kind):
    """With V, W from the tangential solves (exact), the reduced model
    interpolates H along the directions at every solved shift, from the right
    (H b = H_r b) and the left (c^T H = c^T H_r), and matches the bitangential
    derivative c^T H' b = c^T H_r' b (Gugercin, Antoulas & Beattie 2008)."""
    wl = _mimo(e_kind=e_kind)
    rng = np.random.default_rng(5)
    shifts = np.array([0.5, 2.0 + 1.0j, 2.0 - 1.0j, 6.0, 15.0 + 4.0j, 15.0 - 4.0j])
    bt = rng.standard_normal((6, 3)) + 0j
    ct = rng.standard_normal((6, 2)) + 0j
    for i in (1, 4):                      # conjugate directions for conjugate shifts
        bt[i + 1], ct[i + 1] = np.conj(bt[i]), np.conj(ct[i])
    sym = irka._is_symmetric(wl.A, wl.E)
    sV = irka.ReuseSchedule(wl.A, wl.E, transpose=False)
    sW = None if sym else irka.ReuseSchedule(wl.A, wl.E, transpose=True)
    s = shifts
    for z in range(1, 4):
        s, bt, ct, rom, _, _, solved = irka.irka_step_tangential(wl.A, wl.E, wl.B, wl.C, s, bt, ct, sV, sW, z,
                                                                 solver="dense")
        for sig, b, c in zip(solved["sigma"], solved["b"], solved["c"]):
            H, dH = _H_and_dH(wl, sig)
            Hr, dHr = _Hr_and_dHr(rom, sig)
            scale = np.linalg.norm(H)
            assert np.linalg.norm(H @ b - Hr @ b) <= 1e-8 * scale * np.linalg.norm(b)
            assert np.linalg.norm(c @ H - c @ Hr) <= 1e-8 * scale * np.linalg.norm(c)
            d = c @ dH @ b
            assert abs(d - c @ dHr @ b) <= 1e-7 * abs(d)
        # the new shifts are closed under conjugation with conjugate directions
        for i in range(len(s)):
            if s[i].imag > 0:
                assert s[i + 1] == np.conj(s[i])
                np.testing.assert_array_equal(bt[i + 1], np.conj(bt[i]))
                np.testing.assert_array_equal(ct[i + 1], np.conj(ct[i]))


def test_tangential_directions_from_eigenvectors():
    """Line 3 on a pencil with a known eigen-decomposition: A_r = E_r X D X^{-1}
    gives poles D and, up to the scale of each eigenvector, b_i ~ row i of
    X^{-1} E_r^{-1} B_r and c_i ~ column i of C_r^T X; their products c_i b_i^T
    (the residues, independent of the scale) must match exactly."""
    rng = np.random.default_rng(11)
    r, m, q = 5, 3, 2
    X = rng.standard_normal((r, r))
    D = np.array([-1.0, -2.0, -3.5, -5.0, -9.0])
    Er = np.eye(r) + 0.1 * rng.standard_normal((r, r))
    Ar = Er @ X @ np.diag(D) @ np.linalg.inv(X)
    Br = rng.standard_normal((r, m))
    Cr = rng.standard_normal((r, q))
    lam, bt, ct = irka.tangential_directions(Ar, Er, Br, Cr)
    order = np.argsort(lam.real)[::-1]
    lam, bt, ct = lam[order], bt[order], ct[order]
    np.testing.assert_allclose(lam.real, D, rtol=1e-10)
    Binv = np.linalg.solve(X, np.linalg.solve(Er, Br))       # rows: X^{-1} E_r^{-1} B_r
    Cx = Cr.T @ X                                           # columns: C_r^T X
    for i in range(r):
        np.testing.assert_allclose(np.outer(ct[i], bt[i]), np.outer(Cx[:, i], Binv[i]), rtol=1e-8, atol=1e-10)
    # residue form of H_r: sum_i c_i b_i^T / (s - lambda_i)
    s = 0.7 + 2.0j
    Hr = Cr.T @ np.linalg.solve(s * Er - Ar, Br)
    Hres = sum(np.outer(ct[i], bt[i]) / (s - lam[i]) for i in range(r))
    np.testing.assert_allclose(Hres, Hr, rtol=1e-9)


def test_tangential_with_one_input_output_is_siso_irka():
    """m = q = 1: the directions are scalars, the subspaces are the SISO ones,
    so H_r follows the SISO iteration to rounding (1e-12).  The shifts agree
    to 1e-6 only: the scalar directions change the bases (not their spans),
    and the poles of this non-normal reduced pencil move by ~1e-7 under
    that change of basis while H_r does not."""
    wl = W.convdiff3d_siso(N=5)
    res_s = irka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=3, solver="dense")
    r = len(wl.shifts)
    res_t, _ = irka.irka_tangential(wl.A, wl.E, wl.B, wl.C, wl.shifts, np.ones((r, 1)), np.ones((r, 1)), iters=3,
                                    solver="dense")
    for a, b in zip(res_s.shifts_history, res_t.shifts_history):
        np.testing.assert_allclose(a, b, rtol=1e-6)
    w = 1j * np.logspace(0, 4, 50)
    Hs = op.transfer_function_reduced(res_s.Ar, res_s.Er, res_s.Br, res_s.Cr, w)
    Ht = op.transfer_function_reduced(res_t.Ar, res_t.Er, res_t.Br, res_t.Cr, w)
    np.testing.assert_allclose(Ht, Hs, rtol=1e-12)


def test_tangential_iterative_matches_dense():
    """BiCGSTAB with reused SPAI to 1e-8 reproduces the exact tangential
    IRKA's H_r to 1e-6 (MIMO, 3 inputs, 2 outputs)."""
    wl = _mimo(n=120, seed=32)
    r = 6
    shifts = np.array([0.5, 2.0 + 1.0j, 2.0 - 1.0j, 6.0, 15.0 + 4.0j, 15.0 - 4.0j])
    bt = np.ones((r, 3), dtype=complex)
    ct = np.ones((r, 2), dtype=complex)
    rd, _ = irka.irka_tangential(wl.A, wl.E, wl.B, wl.C, shifts, bt, ct, iters=3, solver="dense")
    ri, _ = irka.irka_tangential(wl.A, wl.E, wl.B, wl.C, shifts, bt, ct, iters=3, solver="bicgstab")
    w = 1j * np.logspace(-1, 3, 80)
    H = op.transfer_function(wl.A, wl.E, wl.B, wl.C, w)
    Hd = op.transfer_function_reduced(rd.Ar, rd.Er, rd.Br, rd.Cr, w)
    Hi = op.transfer_function_reduced(ri.Ar, ri.Er, ri.Br, ri.Cr, w)
    err = np.max(np.abs(Hi - Hd), axis=0) / np.max(np.abs(H), axis=0)
    assert np.max(err) <= 1e-6
