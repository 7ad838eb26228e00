"""GPU parity of tangential (MIMO) IRKA, mor_irka_step_tangential, against
the oracle's tangential iteration (Algorithm 2 lines 3-7 with N_j = 0; the
directions of line 3 from the reduced eigenvectors):

  * shift histories within 20 x the oracle's own movement of the shifts when
    its solve tolerance changes from 1e-8 to 1e-10 (at least 1e-6): the IRKA
    fixed-point iteration amplifies solve-level differences;
  * the per-pole residues c_i b_i^T (independent of the eigenvector scale)
    within the same relative bar;
  * H_r on log-spaced frequencies within 1e-6 of the oracle's, relative to
    max |H| per input/output pair (FP64 and mixed precision);
  * m = q = 1 through the tangential entry point reproduces mor_irka_step.
"""
import numpy as np
import pytest

import paper_2003_12759_gb300 as mor
import workloads as W
from oracle import irka as oirka, operator as oop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    mor.load_library()
    hh = mor.mor_create(0)
    yield hh
    mor.mor_destroy(hh)


def _set(h, wl):
    if wl.E is None:
        mor.mor_set_system(h, wl.A, wl.B, wl.C)
    elif isinstance(wl.E, np.ndarray):
        mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E)
    else:
        mor.mor_set_system(h, wl.A, wl.B, wl.C, E=wl.E)


SHIFTS = np.array([0.5, 2.0 + 1.0j, 2.0 - 1.0j, 6.0, 15.0 + 4.0j, 15.0 - 4.0j])


def _start(m, q, seed=7):
    rng = np.random.default_rng(seed)
    bt = rng.standard_normal((6, m)) + 0j
    ct = rng.standard_normal((6, q)) + 0j
    for i in (1, 4):
        bt[i + 1], ct[i + 1] = np.conj(bt[i]), np.conj(ct[i])
    return bt, ct


CASES = {
    "rand_diagE_m3_q2": lambda: W.random_sparse_system(700, 0.006, seed=41, e_kind="diag", m=3, q=2),
    "rand_csrE_m2_q3": lambda: W.random_sparse_system(500, 0.008, seed=42, e_kind="csr", m=2, q=3),
    "convdiff_n512_m4": lambda: W.convdiff3d_mimo(N=8, m=4),
}


def _residues(bt, ct):
    return np.stack([np.outer(c, b) for b, c in zip(bt, ct)])


def _gpu_run(h, wl, iters, opts, bt, ct):
    _set(h, wl)
    s = SHIFTS.copy()
    hist, res = [], []
    rom = None
    for _ in range(iters):
        s, bt, ct, rom, st = mor.mor_irka_step_tangential(h, s, bt, ct, opts)
        hist.append(s.copy())
        res.append(_residues(bt, ct))
        assert st["max_relres"] <= 1.001e-8
    return hist, res, rom


@pytest.mark.parametrize("name", list(CASES))
def test_tangential_irka_matches_oracle(h, name):
    wl = CASES[name]()
    m, q = wl.B.shape[1], wl.C.shape[1]
    bt, ct = _start(m, q)
    iters = 3
    a, used_a = oirka.irka_tangential(wl.A, wl.E, wl.B, wl.C, SHIFTS, bt, ct, iters=iters, tol=1e-8)
    b, _ = oirka.irka_tangential(wl.A, wl.E, wl.B, wl.C, SHIFTS, bt, ct, iters=iters, tol=1e-10)
    move = max(np.max(np.abs(x - y) / np.abs(y)) for x, y in zip(a.shifts_history[1:], b.shifts_history[1:]))
    bar = max(1e-6, 20.0 * move)
    hist, res, rom = _gpu_run(h, wl, iters, mor.mor_default_opts(precision=mor.MOR_FP64), bt, ct)
    for z in range(iters):
        so = a.shifts_history[z + 1]
        assert np.max(np.abs(hist[z] - so) / np.abs(so)) <= bar, (z, hist[z], so, bar)
    # residues of the last iteration's poles
    ro = _residues(a.btil, a.ctil)
    for i in range(len(SHIFTS)):
        assert np.linalg.norm(res[-1][i] - ro[i]) <= max(bar, 1e-6) * 10 * np.linalg.norm(ro[i]), i
    w = np.logspace(-1, 3, 200)
    Hg = mor.mor_eval_tf(h, rom, w)
    Ho = oop.transfer_function_reduced(a.Ar, a.Er, a.Br, a.Cr, 1j * w)
    H = oop.transfer_function(wl.A, wl.E, wl.B, wl.C, 1j * w)
    err = np.max(np.abs(Hg - Ho), axis=0) / np.max(np.abs(H), axis=0)
    assert np.max(err) <= 1e-6, err


def test_tangential_irka_mixed_precision(h):
    wl = CASES["rand_diagE_m3_q2"]()
    bt, ct = _start(3, 2)
    a, _ = oirka.irka_tangential(wl.A, wl.E, wl.B, wl.C, SHIFTS, bt, ct, iters=3, solver="dense")
    _, _, rom = _gpu_run(h, wl, 3, mor.mor_default_opts(), bt, ct)
    w = np.logspace(-1, 3, 200)
    Hg = mor.mor_eval_tf(h, rom, w)
    Ho = oop.transfer_function_reduced(a.Ar, a.Er, a.Br, a.Cr, 1j * w)
    H = oop.transfer_function(wl.A, wl.E, wl.B, wl.C, 1j * w)
    assert np.max(np.max(np.abs(Hg - Ho), axis=0) / np.max(np.abs(H), axis=0)) <= 1e-6


def test_tangential_with_one_input_output_reproduces_siso_step(h):
    wl = W.convdiff3d_siso(N=10)
    r = len(wl.shifts)
    opts = mor.mor_default_opts(precision=mor.MOR_FP64)
    _set(h, wl)
    s1 = wl.shifts.copy()
    for _ in range(2):
        s1, rom1, _ = mor.mor_irka_step(h, s1, opts)
    _set(h, wl)
    s2, bt, ct = wl.shifts.copy(), np.ones((r, 1)), np.ones((r, 1))
    for _ in range(2):
        s2, bt, ct, rom2, _ = mor.mor_irka_step_tangential(h, s2, bt, ct, opts)
    w = np.logspace(0, 5, 300)
    H1 = mor.mor_eval_tf(h, rom1, w)
    H2 = mor.mor_eval_tf(h, rom2, w)
    assert np.max(np.abs(H1 - H2)) <= 1e-7 * np.max(np.abs(H1))
    np.testing.assert_allclose(s2, s1, rtol=1e-4)


def test_siso_step_rejects_mimo_and_tangential_checks_conjugation(h):
    wl = CASES["rand_diagE_m3_q2"]()
    _set(h, wl)
    with pytest.raises(RuntimeError):
        mor.mor_irka_step(h, SHIFTS, mor.mor_default_opts())
    bt, ct = _start(3, 2)
    with pytest.raises(RuntimeError):
        mor.mor_irka_step_tangential(h, SHIFTS[:2], bt[:2], ct[:2], mor.mor_default_opts())
