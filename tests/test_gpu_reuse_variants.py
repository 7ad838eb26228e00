"""GPU parity of the reuse variants of the preconditioner schedule against
the oracle's schedule modes (through the C ABI):

  * MOR_REUSE_FIRST, Table II's first approach along the shifts of an
    iteration (P_i = Q_i P_1, Q_i from min ||A_1 - A_i Q||_F): every shift
    applies the vertical chain plus its own factor;
  * MOR_REUSE_AUTO, Algorithm 4 with the Frobenius-ratio reuse decision
    (reuse when ||A_old - A_new||_F / ||A_old||_F < min(1, ||I - A_new||_F /
    ||I||_F), else a fresh SPAI that restarts the chain).

Checked: the factors the library built in each iteration (read back from its
chains: a fresh SPAI maps a shift to itself, a reuse factor from one shift to
another) against the oracle's build records of the same iteration; H_r on
1000 frequencies within 1e-6 of |H| of the oracle's run; the chains the
first approach applies against the oracle's chains, factor by factor.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_2003_12759_gb300 as mor
import workloads as W
from oracle import irka as oirka, operator as oop, spai as ospai

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    mor.load_library()
    hh = mor.mor_create(0)
    yield hh
    mor.mor_destroy(hh)


def _chain(h, t):
    L, _ = mor.mor_chain_info(h, t)
    out = []
    for i in range(L):
        _, sf, st = mor.mor_get_factor(h, t, i)
        out.append((sf, st))
    return out


@pytest.mark.parametrize("mode,reuse", [("first", mor.MOR_REUSE_FIRST), ("auto", mor.MOR_REUSE_AUTO)])
def test_reuse_variant_builds_and_rom_vs_oracle(h, mode, reuse):
    # 8^3 convection-diffusion, E diagonal, complex shifts from 10 to 1e4: in
    # the first iteration the Frobenius decision rebuilds at the two largest
    # shifts (change ratio above 1), later iterations reuse throughout
    wl = W.convdiff3d_siso(N=8)
    iters = 3
    ref = oirka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=iters, mode=mode)
    mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E)
    opts = mor.mor_default_opts(precision=mor.MOR_FP64, reuse=reuse)
    s = wl.shifts.copy()
    rom = None
    # oracle records of the primal operator, per iteration
    nrec = len(ref.builds) // 2          # primal records first, then the transposed ones
    prim = ref.builds[:nrec]
    for z in range(1, iters + 1):
        solved = oirka.solve_shifts_of(s)
        s, rom, st = mor.mor_irka_step(h, s, opts)
        recs = [r for r in prim if r[0] == z]
        assert st["max_relres"] <= 1.001e-8
        if len(recs) != st["nsolve"]:
            # the two runs' shifts split differently into conjugate pairs and real
            # shifts (a pair with a small imaginary part turning real): no record match
            assert z > 1
            continue
        chain = _chain(h, 0)
        # the iteration's factors are the last len(recs) - 1 horizontal ones plus the vertical one
        horiz = chain[len(chain) - (len(recs) - 1):] if len(recs) > 1 else []
        vert = chain[len(chain) - len(recs)]
        kind_v = "spai" if vert[0] == vert[1] else "vertical"
        assert kind_v == recs[0][2], (z, kind_v, recs[0])
        assert np.isclose(vert[1], solved[0], rtol=1e-9)
        for i, (f, rec) in enumerate(zip(horiz, recs[1:]), start=1):
            if mode == "first":
                assert rec[2] == "first" and np.isclose(f[0], solved[0], rtol=1e-9), (z, i, f, rec)
            else:
                kind = "spai" if f[0] == f[1] else "horizontal"
                assert kind == rec[2], (z, i, f, rec)
                if kind == "horizontal":
                    assert np.isclose(f[0], solved[i - 1], rtol=1e-9)
            assert np.isclose(f[1], solved[i], rtol=1e-9)
        n_spai = sum(1 for r in recs if r[2] == "spai")
        assert st["builds_spai"] == 2 * n_spai and st["builds_reuse"] == 2 * (len(recs) - n_spai), (z, st)
    w = 1j * np.logspace(0, 5, 1000)
    Ar, Er, Br, Cr = rom.arrays()
    Hg = oop.transfer_function_reduced(Ar, Er, Br, Cr, w)[:, 0, 0]
    Ho = oop.transfer_function_reduced(ref.Ar, ref.Er, ref.Br, ref.Cr, w)[:, 0, 0]
    H = oop.transfer_function(wl.A, wl.E, wl.B, wl.C, w)[:, 0, 0]
    assert np.max(np.abs(Hg - Ho) / np.abs(H)) <= 1e-6


def test_auto_reuse_decisions_in_first_iteration(h):
    """The decision of the first iteration (identical shifts on both sides) is
    the oracle's exactly: fresh SPAIs at the two largest shifts."""
    wl = W.convdiff3d_siso(N=8)
    ref = oirka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=1, mode="auto")
    kinds = [r[2] for r in ref.builds[: len(ref.builds) // 2]]
    assert kinds.count("spai") >= 2          # the workload exercises both branches
    mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E)
    mor.mor_irka_step(h, wl.shifts.copy(), mor.mor_default_opts(precision=mor.MOR_MIXED, reuse=mor.MOR_REUSE_AUTO))
    chain = _chain(h, 0)
    got = ["spai" if a == b else "horizontal" for a, b in chain]
    assert got == kinds


def test_first_approach_chains_apply_like_the_oracle(h):
    """With the first approach, shift i applies P_1 then its own Q_i: the
    library's preconditioner for each shift equals the oracle's chain (FP64
    factors from independent least-squares solves: 1e-8 relative)."""
    wl = W.convdiff3d_siso(N=9)
    s_solve = oirka.solve_shifts_of(wl.shifts)
    mor.mor_set_system(h, wl.A, wl.B, wl.C, E_diag=wl.E)
    opts = mor.mor_default_opts(precision=mor.MOR_FP64, reuse=mor.MOR_REUSE_FIRST)
    mor.mor_irka_step(h, wl.shifts.copy(), opts)
    sched = oirka.ReuseSchedule(wl.A, wl.E, transpose=False, mode="first")
    chains = sched.chains(1, s_solve)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(wl.n) + 1j * rng.standard_normal(wl.n)
    lib_chain = _chain(h, 0)
    assert len(lib_chain) == len(s_solve)    # P_1 and one Q per further shift
    for i, s in enumerate(s_solve):
        # the library's factor i (i >= 1) maps s_1 to s_i; apply P_1 then that factor
        y0 = mor.mor_apply_precond(h, [s_solve[0]], x[:, None])[:, 0]
        ref = ospai.chain_apply(chains[i], x)
        if i == 0:
            assert np.linalg.norm(y0 - ref) <= 1e-9 * np.linalg.norm(ref)
            continue
        vals, sf, st = mor.mor_get_factor(h, 0, i)
        rowptr, col = mor.mor_get_pattern(h, 0)
        Q = sp.csr_matrix((vals, col, rowptr), shape=(wl.n, wl.n))
        assert np.isclose(sf, s_solve[0]) and np.isclose(st, s)
        y = Q @ y0
        assert np.linalg.norm(y - ref) <= 1e-8 * np.linalg.norm(ref), i
