"""Pins of the oracle's grid-map form of the ligand-pocket terms: grid-point values equal
the direct one-atom energy, the interpolation equals scipy's regular-grid linear
interpolation of the corner energies, the interpolated gradient matches central
differences inside a cell, the error shrinks as O(h^2), and atoms outside the domain
keep the direct sum."""
import math

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

from paper_2510_24186_b300 import synth


def vina(orc):
    return orc.make_params(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)


def trids1(orc):
    rng = np.random.default_rng(3)
    g = np.zeros((8, 8, 2, 3))
    g[..., 0] = rng.uniform(0.2, 1.0, (8, 8, 2))
    g[..., 1] = rng.uniform(2.0, 4.5, (8, 8, 2))
    g[..., 2] = rng.uniform(0.4, 1.2, (8, 8, 2))
    return orc.make_params(1, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, 10.0, gmm=g)


def one_atom(orc, ti):
    st, lg = orc.pack(np.zeros((1, 3)), [ti], np.zeros((0, 2)), [])
    return lg


def at(x):
    return np.array([x[0], x[1], x[2], 1, 0, 0, 0.0])


@pytest.fixture(scope="module")
def pocket():
    w = synth.workload("single_ligand")
    return w.pocket


@pytest.mark.parametrize("mk", [vina, trids1])
def test_map_value_at_grid_points_is_the_direct_energy(orc, pocket, mk):
    p = mk(orc)
    mp = orc.maps((-6.0, -6.0, -6.0), 0.5, (25, 25, 25))
    rng = np.random.default_rng(1)
    for _ in range(20):
        ti = int(rng.integers(0, 8))
        lg = one_atom(orc, ti)
        g = -6.0 + 0.5 * rng.integers(1, 23, 3)
        _, ev_m = orc.score(p, pocket.xyz, pocket.type, lg, at(g), mp=mp)
        _, ev_d = orc.score(p, pocket.xyz, pocket.type, lg, at(g))
        assert ev_m.n_map_atoms == 1
        assert ev_m.e_total == pytest.approx(ev_d.e_total, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("mk", [vina, trids1])
def test_interpolation_matches_scipy_regular_grid(orc, pocket, mk):
    """Corner energies from the direct path; scipy's linear interpolation on the 2x2x2
    corner grid gives the value and (by differences of interpolants) the gradient."""
    p = mk(orc)
    h = 0.4
    lo = np.array([-7.0, -5.0, -6.0])
    mp = orc.maps(lo, h, (30, 30, 30))
    rng = np.random.default_rng(2)
    for _ in range(15):
        ti = int(rng.integers(0, 8))
        lg = one_atom(orc, ti)
        c = rng.integers(2, 26, 3)
        f = rng.uniform(0.05, 0.95, 3)
        x = lo + h * (c + f)
        V = np.zeros((2, 2, 2))
        for a in range(2):
            for b in range(2):
                for k in range(2):
                    g = lo + h * (c + np.array([a, b, k]))
                    V[a, b, k] = orc.score(p, pocket.xyz, pocket.type, lg, at(g))[1].e_total
        axes = [lo[d] + h * np.array([c[d], c[d] + 1]) for d in range(3)]
        interp = RegularGridInterpolator(axes, V, method="linear")
        _, ev = orc.score(p, pocket.xyz, pocket.type, lg, at(x), mp=mp)
        assert ev.e_total == pytest.approx(float(interp(x)[0]), rel=1e-11, abs=1e-11)
        # the interpolant is linear along each axis inside the cell: its derivative is the
        # difference of the values on the two faces over h
        for d in range(3):
            x0, x1 = x.copy(), x.copy()
            x0[d], x1[d] = axes[d][0], axes[d][1]
            gd = (float(interp(x1)[0]) - float(interp(x0)[0])) / h
            assert ev.g_dof[d] == pytest.approx(gd, rel=1e-9, abs=1e-9)


def test_interpolated_gradient_matches_central_differences(orc, pocket):
    p = vina(orc)
    mp = orc.maps((-9.0, -9.0, -9.0), 0.375, (50, 50, 50))
    w = synth.workload("single_ligand")
    lig = w.ligands[0]
    st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(4):
        q = rng.normal(size=4)
        dof = np.concatenate([rng.uniform(-2, 2, 3), q / np.linalg.norm(q), rng.uniform(-math.pi, math.pi, lg.n_tor)])
        _, ev = orc.score(p, pocket.xyz, pocket.type, lg, dof, mp=mp)
        assert ev.n_map_atoms == lg.n_atoms
        for j in range(7 + lg.n_tor):
            def fd(hh):
                dp, dm = dof.copy(), dof.copy()
                dp[j] += hh
                dm[j] -= hh
                return (orc.score(p, pocket.xyz, pocket.type, lg, dp, mp=mp)[1].e_total
                        - orc.score(p, pocket.xyz, pocket.type, lg, dm, mp=mp)[1].e_total) / (2 * hh)
            f1, f2 = fd(1e-6), fd(5e-7)
            if abs(f1 - f2) > 1e-4 * (1 + abs(f1)):   # an atom crossed a cell face
                continue
            assert f2 == pytest.approx(ev.g_dof[j], rel=1e-5, abs=1e-6), j
            checked += 1
    assert checked > 20


def test_map_error_shrinks_quadratically_with_spacing(orc, pocket):
    p = vina(orc)
    rng = np.random.default_rng(7)
    pts = [rng.uniform(-4, 4, 3) for _ in range(30)]
    errs = []
    for h in (0.4, 0.2, 0.1):
        n = int(round(20 / h)) + 1
        mp = orc.maps((-10.0, -10.0, -10.0), h, (n, n, n))
        e = 0.0
        for k, x in enumerate(pts):
            lg = one_atom(orc, k % 8)
            em = orc.score(p, pocket.xyz, pocket.type, lg, at(x), mp=mp)[1].e_total
            ed = orc.score(p, pocket.xyz, pocket.type, lg, at(x))[1].e_total
            e = max(e, abs(em - ed))
        errs.append(e)
    assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1]


def test_atoms_outside_the_domain_keep_the_direct_sum(orc, pocket):
    p = vina(orc)
    mp = orc.maps((-2.0, -2.0, -2.0), 0.5, (9, 9, 9))   # covers [-2, 2]^3
    rng = np.random.default_rng(9)
    for x in ([2.5, 0, 0], [0, -2.3, 0], [1.999, 1.0, 5.0], [-3.0, -3.0, -3.0]):
        lg = one_atom(orc, int(rng.integers(0, 8)))
        _, em = orc.score(p, pocket.xyz, pocket.type, lg, at(np.array(x)), mp=mp)
        _, ed = orc.score(p, pocket.xyz, pocket.type, lg, at(np.array(x)))
        assert em.n_map_atoms == 0
        assert em.e_total == ed.e_total
