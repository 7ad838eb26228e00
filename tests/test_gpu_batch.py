"""GPU parity of the batched uneven systems path (independent systems of
different sizes, all shifts and systems advancing in the same launches),
against the CPU oracle run system by system.

Bars: every (system, shift) solution reaches the true relative residual 1e-8
of its own system (recomputed by the oracle in FP64), and in FP64 mode the
BiCGSTAB iteration counts, run system by system in the oracle, match: the
total over all (system, shift) pairs within 10%, each pair within max(3,
25%) (individual counts of ill-conditioned solves move with the summation
order of the dot products; a 64-vs-53 pair was observed on a sigma = 1
Laplacian) -- the batch must not couple the systems' Krylov iterations,
which would change the counts far more."""
import numpy as np
import pytest

import paper_2003_12759_gb300 as mor
import workloads as W
from oracle import operator as oop, spai as ospai, krylov as okry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    mor.load_library()
    hh = mor.mor_create(0)
    yield hh
    mor.mor_destroy(hh)


def _batch(nsys=6, seed=7):
    # the uneven-batch generator at small sizes (n_s in [300, 2500])
    return W.uneven_laplace2d_batch(num_systems=nsys, n_lo=300, n_hi=2500, seed=seed)


@pytest.mark.parametrize("precision", [mor.MOR_FP64, mor.MOR_MIXED])
@pytest.mark.parametrize("transpose", [0, 1])
def test_batch_solves_match_per_system_oracle(h, precision, transpose):
    sysl = _batch()
    mor.mor_set_batch(h, [w.A for w in sysl], [w.B[:, 0] for w in sysl], [w.C[:, 0] for w in sysl])
    nsys, off = mor.mor_batch_info(h)
    assert nsys == len(sysl) and off[-1] == sum(w.n for w in sysl)
    shifts = [1.0, 10.0, 100.0, 1000.0 + 50.0j]
    mor.mor_build_precond(h, shifts[0], transpose, precision)
    for s in shifts[1:]:
        mor.mor_update_precond(h, s, transpose)
    X, stats, code = mor.mor_batch_solve(h, shifts, transpose, mor.mor_default_opts(precision=precision))
    assert code == mor.MOR_OK
    counts = []
    for i, w in enumerate(sysl):
        xs = X[off[i]:off[i + 1]]
        b = (w.C if transpose else w.B)[:, 0]
        S = ospai.spai_pattern(w.A, w.E, transpose=bool(transpose))
        Ms = [oop.A_sigma(w.A, w.E, s, transpose=bool(transpose)) for s in shifts]
        F = [ospai.spai(Ms[0], S)] + [ospai.reuse_factor(Ms[j - 1], Ms[j], S) for j in range(1, len(shifts))]
        for c, s in enumerate(shifts):
            rel = np.linalg.norm(b - Ms[c] @ xs[:, c]) / np.linalg.norm(b)
            assert rel <= 1.001e-8, (i, c, rel)
            assert stats[i][c]["status"] == mor.MOR_OK
            if precision == mor.MOR_FP64:
                _, ito, _, _ = okry.bicgstab(lambda v, M=Ms[c]: M @ v,
                                             lambda v, f=F[: c + 1]: ospai.chain_apply(f, v),
                                             b.astype(Ms[c].dtype), tol=1e-8)
                counts.append((i, c, stats[i][c]["iters"], ito))
    if counts:
        tg = sum(x[2] for x in counts)
        to = sum(x[3] for x in counts)
        assert abs(tg - to) <= 0.1 * to, counts
        for (i, c, itg, ito) in counts:
            assert abs(itg - ito) <= max(3, 0.25 * ito), counts


def test_batch_unpreconditioned_and_single_system_equivalence(h):
    """A one-system batch solves exactly like mor_set_system + mor_solve_shifts."""
    w = _batch(1, seed=3)[0]
    shifts = [5.0, 50.0]
    opts = mor.mor_default_opts(precision=mor.MOR_FP64, precond=2)
    mor.mor_set_batch(h, [w.A], [w.B[:, 0]], [w.C[:, 0]])
    Xb, sb, cb = mor.mor_batch_solve(h, shifts, 0, opts)
    mor.mor_set_system(h, w.A, w.B, w.C)
    Xs, ss, cs = mor.mor_solve_shifts(h, shifts, 0, opts)
    assert cb == cs == mor.MOR_OK
    assert [x["iters"] for x in sb[0]] == [x["iters"] for x in ss]
    np.testing.assert_allclose(Xb, Xs, rtol=1e-12, atol=1e-14 * np.abs(Xs).max())


def test_batch_failed_mixed_columns_fall_back_to_fp64(h):
    """In a batch of systems a column (shift) that fails in mixed precision in
    any system is solved again in FP64 for every system; all reach 1e-8."""
    sysl = _batch()
    mor.mor_set_batch(h, [w.A for w in sysl], [w.B[:, 0] for w in sysl], [w.C[:, 0] for w in sysl])
    nsys, off = mor.mor_batch_info(h)
    shifts = [1.0, 10.0, 100.0]
    mor.mor_build_precond(h, shifts[0], 0, mor.MOR_MIXED)
    for s in shifts[1:]:
        mor.mor_update_precond(h, s, 0)
    weak = dict(max_refine=1, inner_tol=1e-3)
    _, st0, code0 = mor.mor_batch_solve(h, shifts, 0, mor.mor_default_opts(fp64_fallback=0, **weak))
    assert code0 == mor.MOR_ENOCONV
    X, st1, code1 = mor.mor_batch_solve(h, shifts, 0, mor.mor_default_opts(**weak))
    assert code1 == mor.MOR_OK
    for i, w in enumerate(sysl):
        b = w.B[:, 0]
        for c, s in enumerate(shifts):
            assert st1[i][c]["fallback"] == 1 and st1[i][c]["status"] == mor.MOR_OK
            rel = np.linalg.norm(b - oop.A_sigma(w.A, w.E, s) @ X[off[i]:off[i + 1], c]) / np.linalg.norm(b)
            assert rel <= 1.001e-8, (i, c, rel)


def test_batch_of_equal_systems_in_the_diagonal_layout(h):
    """A batch of equal 2D Laplacians (the block-diagonal pattern has 5
    diagonals, with padding where a diagonal crosses from one system into the
    next) stored in the diagonal layout: every (system, shift) solution at the
    1e-8 true residual of its own system, and the same iterations and
    solutions as the CSR layout."""
    sysl = [W.laplace2d_siso(N=20, seed=s) for s in range(4)]
    shifts = [2.0, 20.0, 200.0 + 10.0j]
    out = {}
    for fmt in (mor.MOR_FMT_CSR, mor.MOR_FMT_DIA):
        mor.mor_set_batch(h, [w.A for w in sysl], [w.B[:, 0] for w in sysl], [w.C[:, 0] for w in sysl], fmt=fmt)
        assert mor.mor_get_info(h)["format"] == fmt
        nsys, off = mor.mor_batch_info(h)
        mor.mor_build_precond(h, shifts[0], 0, mor.MOR_MIXED)
        for s in shifts[1:]:
            mor.mor_update_precond(h, s, 0)
        X, stats, code = mor.mor_batch_solve(h, shifts, 0, mor.mor_default_opts(precision=mor.MOR_MIXED))
        assert code == mor.MOR_OK
        for i, w in enumerate(sysl):
            xs = X[off[i]:off[i + 1]]
            b = w.B[:, 0]
            for c, s in enumerate(shifts):
                M = oop.A_sigma(w.A, w.E, s)
                assert np.linalg.norm(b - M @ xs[:, c]) <= 1.001e-8 * np.linalg.norm(b), (fmt, i, c)
        out[fmt] = (X, [[x["iters"] for x in st] for st in stats])
    (Xc, ic), (Xd, idg) = out[mor.MOR_FMT_CSR], out[mor.MOR_FMT_DIA]
    assert ic == idg
    np.testing.assert_allclose(Xd, Xc, rtol=0, atol=1e-12 * np.abs(Xc).max())
