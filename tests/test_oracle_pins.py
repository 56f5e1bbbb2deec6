"""Pins for the FP64 oracle: closed forms, invariants and published values.

None of these retypes the oracle's formula: each compares it with a result fixed by the
physics or the mathematics (a closed-form field or trajectory, a conservation law, a
symmetry) or with a value printed in the paper or in CODATA 2018.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2502_10640_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CODATA = json.load(open(os.path.join(GOLD, "codata2018.json")))
C_LIGHT = CODATA["speed_of_light_m_per_s"]["value"]
R_E = CODATA["classical_electron_radius_m"]["value"]
E_OVER_M = CODATA["electron_charge_to_mass_C_per_kg"]["value"]
# k e^2 / m_e from the oracle's constants; the constants themselves are pinned to the
# classical electron radius and the specific charge in test_constants_match_codata_derived_values,
# so the closed-form tests below can use a tight tolerance.
_C = oracle.constants()
KE2_M = _C["k"] * _C["e"] ** 2 / _C["me"]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# --- constants ---------------------------------------------------------------------------

def test_constants_match_codata_derived_values():
    c = oracle.constants()
    assert c["e"] == CODATA["elementary_charge_C"]["value"]
    r_e = c["k"] * c["e"] ** 2 / (c["me"] * C_LIGHT ** 2)
    assert abs(r_e / R_E - 1) < 3 * CODATA["classical_electron_radius_m"]["rel_unc"]
    assert abs(c["e"] / c["me"] / E_OVER_M - 1) < 3 * CODATA["electron_charge_to_mass_C_per_kg"]["rel_unc"]


# --- fields: closed forms ----------------------------------------------------------------

@pytest.mark.parametrize("eps", [0.0, 0.3e-6])
def test_two_body_acceleration_closed_form(eps):
    d, w0, w1 = 1.7e-6, 3.0, 5.0
    pos = np.array([[-d / 2, 0.2e-6, 0.0], [d / 2, 0.2e-6, 0.0]])
    a = oracle.accel(pos, np.array([w0, w1]), eps)
    # repulsion along the line: particle 0 is pushed to -x by particle 1 (weight w1)
    mag0 = KE2_M * w1 * d / (d * d + eps * eps) ** 1.5
    mag1 = KE2_M * w0 * d / (d * d + eps * eps) ** 1.5
    np.testing.assert_allclose(a[0], [-mag0, 0, 0], rtol=1e-12, atol=1e-12 * mag0)
    np.testing.assert_allclose(a[1], [+mag1, 0, 0], rtol=1e-12, atol=1e-12 * mag1)
    # the field of negative charges points toward them: E0 along +x
    E = oracle.fields(pos, np.array([w0, w1]), eps)
    assert E[0, 0] > 0 and E[1, 0] < 0
    np.testing.assert_allclose(E[0, 0] * (-E_OVER_M), a[0, 0], rtol=1e-9)


def test_ring_on_axis_field():
    """n equal charges on a ring of radius rho: field on the axis is k Q z / (z^2+rho^2)^(3/2)."""
    n, rho, z, w = 7, 2.0e-6, 1.3e-6, 4.0
    ang = 2 * np.pi * np.arange(n) / n
    ring = np.stack([rho * np.cos(ang), rho * np.sin(ang), np.zeros(n)], axis=1)
    pos = np.vstack([ring, [[0.0, 0.0, z]]])
    wts = np.array([w] * n + [1.0])
    a = oracle.accel(pos, wts, 0.0)
    expect_z = KE2_M * n * w * z / (z * z + rho * rho) ** 1.5
    assert abs(a[-1, 2] / expect_z - 1) < 1e-12
    assert abs(a[-1, 0]) < 1e-12 * expect_z and abs(a[-1, 1]) < 1e-12 * expect_z


def test_regular_tetrahedron():
    """Each vertex is pushed radially out with |a| = sqrt(6) k e^2 w / (m_e a^2)."""
    edge, w = 3.0e-6, 2.5
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    v *= edge / (2 * math.sqrt(2))           # edge length of this set is 2 sqrt(2)
    centre = np.array([0.4e-6, -1.0e-6, 2.0e-6])
    pos = v + centre
    a = oracle.accel(pos, w, 0.0)
    mag = math.sqrt(6) * KE2_M * w / edge ** 2
    for i in range(4):
        u = v[i] / np.linalg.norm(v[i])
        np.testing.assert_allclose(a[i], mag * u, rtol=1e-12, atol=1e-12 * mag)


def test_uniform_sphere_interior_field_slope():
    """Inside a uniform ball a_r = K r with K = k e^2 N w / (m_e R^3), up to sampling noise."""
    n, R, w = 8000, 20e-6, 3.0
    pos = wl.uniform_sphere(n, R, seed=11)
    a = oracle.accel(pos, w, 0.0)
    r = np.linalg.norm(pos, axis=1)
    ar = np.einsum("ij,ij->i", a, pos) / r
    inner = r < 0.7 * R
    slope = np.sum(ar[inner] * r[inner]) / np.sum(r[inner] ** 2)
    K = KE2_M * n * w / R ** 3
    assert abs(slope / K - 1) < 0.02, slope / K


def test_shell_theorem_exterior_point():
    """A probe far outside a uniform ball feels k Q / r^2 directed radially."""
    n, R, w = 8000, 20e-6, 3.0
    ball = wl.uniform_sphere(n, R, seed=12)
    probe = np.array([[0.0, 3.0 * R, 0.0]])
    pos = np.vstack([ball, probe])
    wts = np.concatenate([np.full(n, w), [1e-30]])       # negligible back-reaction
    a = oracle.accel(pos, wts, 0.0)[-1]
    expect = KE2_M * n * w / (3.0 * R) ** 2
    assert abs(a[1] / expect - 1) < 0.01
    assert math.hypot(a[0], a[2]) < 0.01 * expect


# --- fields: brute force in exact arithmetic ------------------------------------------------

def _exact_fields(pos, w, eps, k, qe):
    """Eq. B / Eq. E recomputed without rounding error in the geometry: every double is
    taken as the exact rational it represents, the separations and s = |d|^2 + eps^2 are
    exact fractions, and only s^(3/2) and the quotient are rounded, in 60-digit decimal
    arithmetic (correctly rounded square root).  Returns the field [N][3] and, per
    component, sum_j |Q_j d / s^(3/2)| (the scale of the summation error bound)."""
    import decimal
    from fractions import Fraction
    ctx = decimal.Context(prec=60)
    dec = lambda f: ctx.divide(decimal.Decimal(f.numerator), decimal.Decimal(f.denominator))
    n = pos.shape[0]
    P = [[Fraction(float(x)) for x in row] for row in pos]
    W = [Fraction(float(x)) for x in np.broadcast_to(w, (n,))]
    e2 = Fraction(float(eps)) ** 2
    kq = dec(Fraction(float(k)) * Fraction(float(qe)))
    E = np.zeros((n, 3))
    S = np.zeros((n, 3))
    for i in range(n):
        acc = [decimal.Decimal(0)] * 3
        mag = [decimal.Decimal(0)] * 3
        for j in range(n):
            if j == i:
                continue
            d = [P[i][c] - P[j][c] for c in range(3)]
            s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + e2
            if s == 0:
                continue
            sd = dec(s)
            s32 = ctx.multiply(sd, sd.sqrt(ctx))
            for c in range(3):
                t = ctx.divide(dec(W[j] * d[c]), s32)
                acc[c] = ctx.add(acc[c], t)
                mag[c] = ctx.add(mag[c], abs(t))
        for c in range(3):
            E[i, c] = float(ctx.multiply(kq, acc[c]))
            S[i, c] = float(abs(ctx.multiply(kq, mag[c])))
    return E, S


@pytest.mark.parametrize("n", [2, 5, 17, 64])
@pytest.mark.parametrize("eps_frac", [0.0, 0.3])
def test_brute_force_exact_fields_small_n(n, eps_frac):
    """Random clouds of N <= 64 with random weights: the oracle's field equals the field
    recomputed in exact arithmetic to the FP64 rounding of its own sum (per element within
    the recursive-summation bound 4 (N + 4) u sum_j |term|, and 1e-14 in relative L2)."""
    sigma = 2e-6
    pos = wl.gaussian_bunch(n, sigma, seed=500 + n)
    w = 1.0 + 4.0 * wl.uniform(500 + n, 9, n)
    eps = eps_frac * sigma
    c = oracle.constants()
    E = oracle.fields(pos, w, eps)
    ref, scale = _exact_fields(pos, w, eps, c["k"], -c["e"])
    u = 2.0 ** -53
    assert np.all(np.abs(E - ref) <= 4 * (n + 4) * u * scale + 1e-300)
    assert rel(E, ref) <= 1e-14


# --- fields: invariants ------------------------------------------------------------------

def _random_cloud(n, seed, scale=5e-6):
    pos = wl.gaussian_bunch(n, scale, seed)
    w = 1.0 + wl.uniform(seed, 9, n) * 4.0
    return pos, w


def test_third_law_net_force_vanishes():
    pos, w = _random_cloud(600, 21)
    E = oracle.fields(pos, w, 1e-8)
    F = w[:, None] * E                 # force up to the factor q_e
    assert np.linalg.norm(F.sum(axis=0)) < 1e-13 * np.abs(F).sum()


def test_permutation_equivariance():
    pos, w = _random_cloud(300, 22)
    perm = np.argsort(wl.uniform(22, 10, 300))
    E = oracle.fields(pos, w, 0.0)
    Ep = oracle.fields(pos[perm], w[perm], 0.0)
    assert rel(Ep, E[perm]) < 1e-13


def test_translation_rotation_scaling_linearity():
    pos, w = _random_cloud(300, 23)
    eps = 2e-8
    E = oracle.fields(pos, w, eps)
    # translation
    assert rel(oracle.fields(pos + np.array([1e-5, -3e-5, 2e-5]), w, eps), E) < 1e-8
    # rotation about an arbitrary axis
    th = 0.7
    axis = np.array([1.0, 2.0, -0.5]); axis /= np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    Rm = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    assert rel(oracle.fields(pos @ Rm.T, w, eps), E @ Rm.T) < 1e-12
    # scaling: r -> lam r, eps -> lam eps gives E -> E / lam^2
    lam = 3.0
    assert rel(oracle.fields(lam * pos, w, lam * eps), E / lam ** 2) < 1e-13
    # linear in the source weights
    assert rel(oracle.fields(pos, 2.5 * w, eps), 2.5 * E) < 1e-14


def test_cube_lattice_symmetries():
    pos = wl.cube_lattice(8, 1e-4)
    n = pos.shape[0]
    E = oracle.fields(pos, 1.0, 0.0)
    scale = np.abs(E).max()
    # inversion through the centre maps lattice point i to n-1-i
    assert np.abs(E + E[::-1]).max() < 1e-12 * scale
    # mirror x -> -x maps (a, b, c) to (7-a, b, c)
    idx = np.arange(n).reshape(8, 8, 8)
    mirror = idx[::-1, :, :].ravel()
    Em = E[mirror] * np.array([-1.0, 1.0, 1.0])
    assert np.abs(E - Em).max() < 1e-12 * scale
    # outward on the whole surface layer: x component has the sign of x at the +-x faces
    face = np.abs(pos[:, 0]) > 0.4e-4
    assert np.all(np.sign(-E[face, 0]) == np.sign(pos[face, 0]))  # a = -|e|/m E points outward


def test_single_particle_and_coincident_pairs():
    assert np.all(oracle.fields(np.array([[1e-6, 2e-6, 3e-6]]), 1.0, 0.0) == 0.0)
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1e-6, 0.0, 0.0]])
    E = oracle.fields(pos, 1.0, 0.0)
    assert np.all(np.isfinite(E))
    # the coincident pair contributes nothing: particles 0 and 1 see only particle 2
    np.testing.assert_allclose(E[0], E[1], rtol=0, atol=0)
    np.testing.assert_allclose(np.abs(E[0, 0]) * 2, np.abs(E[2, 0]), rtol=1e-14)


def test_fields_subset_rows_follow_index():
    pos, w = _random_cloud(200, 24)
    E = oracle.fields(pos, w, 1e-8)
    idx = np.array([199, 3, 3, 0, 117])
    np.testing.assert_array_equal(oracle.fields_subset(pos, w, 1e-8, idx), E[idx])


# --- potential energy ----------------------------------------------------------------------

def test_potential_energy_closed_forms():
    c = oracle.constants()
    ke2 = c["k"] * c["e"] ** 2
    d, w0, w1 = 2e-6, 3.0, 7.0
    pos = np.array([[0, 0, 0], [d, 0, 0]], dtype=float)
    assert abs(oracle.potential_energy(pos, np.array([w0, w1]), 0.0) / (ke2 * w0 * w1 / d) - 1) < 1e-14
    eps = 0.5e-6
    assert abs(oracle.potential_energy(pos, np.array([w0, w1]), eps)
               / (ke2 * w0 * w1 / math.sqrt(d * d + eps * eps)) - 1) < 1e-14
    edge = 1e-6
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) * edge / (2 * math.sqrt(2))
    assert abs(oracle.potential_energy(v, 2.0, 0.0) / (6 * ke2 * 4.0 / edge) - 1) < 1e-13


# --- diagnostics -----------------------------------------------------------------------------

def test_diagnostics_hand_values():
    c = oracle.constants()
    # off-centre in x so that raw (Eq. I) and centred moments differ
    pos = np.array([[3.0, 0, 0], [1.0, 0, 0], [2.0, 2.0, 0], [2.0, -2.0, 0]]) * 1e-6
    vel = np.array([[1.0, 0, 0], [1.0, 0, 0], [0, 3.0, 0], [0, -3.0, 0]]) * 1e3
    w = np.array([1.0, 2.0, 3.0, 4.0])
    d = oracle.diagnostics(pos, vel, w)
    assert abs(d["cx"] - 2e-6) < 1e-21 and d["cy"] == 0.0
    assert abs(d["rms_radius"] / (math.sqrt(2.5) * 1e-6) - 1) < 1e-14
    assert abs(d["ke"] / (0.5 * c["me"] * (1 * 1 + 2 * 1 + 3 * 9 + 4 * 9) * 1e6) - 1) < 1e-14
    assert abs(d["px"] / (c["me"] * 3e3) - 1) < 1e-14
    assert abs(d["py"] / (c["me"] * (9 - 12) * 1e3) - 1) < 1e-14
    assert d["pz"] == 0.0
    # raw moments: <x^2> = 4.5e-12, <vx^2> = 0.5e6, <x vx> = 1e-3 -> emit^2 = 1.25e-6
    assert abs(d["emit_x"] / math.sqrt(1.25e-6) - 1) < 1e-12
    assert abs(d["x_rms"] / (math.sqrt(4.5) * 1e-6) - 1) < 1e-14
    assert d["x_max"] == 3e-6 and d["vx_max"] == 1e3
    assert abs(d["vx_rms"] / math.sqrt(0.5e6) - 1) < 1e-14


def test_emittance_vanishes_for_linear_phase_space():
    x = wl.gaussian(31, 0, 500) * 1e-5
    pos = np.stack([x, np.zeros_like(x), np.zeros_like(x)], axis=1)
    vel = 3.7e7 * pos                              # v_x proportional to x: a line in phase space
    d = oracle.diagnostics(pos, vel, 1.0)
    scale = d["x_rms"] * d["vx_rms"]
    assert d["emit_x"] <= 1e-7 * scale


# --- integrator ------------------------------------------------------------------------------

def _two_body_separation_closed_form(t, r0, C):
    """Separation u r0 at time t for two like charges released at rest (energy integral)."""
    tau = math.sqrt(r0 ** 3 / C)

    def t_of_u(u):
        return tau * (math.sqrt(u * (u - 1)) + math.log(math.sqrt(u) + math.sqrt(u - 1)))
    if t == 0:
        return r0
    u = brentq(lambda u: t_of_u(u) - t, 1.0, 1e6, xtol=1e-15, rtol=1e-15)
    return u * r0


def _two_body_error(nsteps, w=2.0, r0=1e-6, u_end=3.0):
    C = 4 * KE2_M * w
    tau = math.sqrt(r0 ** 3 / C)
    T = tau * (math.sqrt(u_end * (u_end - 1)) + math.log(math.sqrt(u_end) + math.sqrt(u_end - 1)))
    pos = np.array([[-r0 / 2, 0, 0], [r0 / 2, 0, 0]])
    vel = np.zeros((2, 3))
    p, v, a = oracle.vv_run(pos, vel, None, w, 0.0, T / nsteps, nsteps)
    sep = p[1, 0] - p[0, 0]
    exact = _two_body_separation_closed_form(T, r0, C)
    return abs(sep - exact) / exact, p, v


def test_two_electron_separation_second_order():
    e1, _, _ = _two_body_error(100)
    e2, _, _ = _two_body_error(200)
    e3, _, _ = _two_body_error(400)
    assert e3 < 2e-5
    for lo, hi in ((e1, e2), (e2, e3)):
        assert 3.2 < lo / hi < 4.8, (e1, e2, e3)


def test_two_electron_energy_and_momentum():
    w, r0 = 2.0, 1e-6
    _, p, v = _two_body_error(400, w=w, r0=r0)
    d = oracle.diagnostics(p, v, w)
    pe0 = oracle.potential_energy(np.array([[0, 0, 0], [r0, 0, 0]], float), w, 0.0)
    tot = d["ke"] + oracle.potential_energy(p, w, 0.0)
    assert abs(tot / pe0 - 1) < 1e-5
    assert abs(d["px"]) < 1e-12 * d["ke"] / np.abs(v).max()


@pytest.mark.slow
def test_cold_uniform_sphere_explosion_homologous():
    """R_rms(t)/R_rms(0) follows the shell ODE s'' = K / s^2 of a cold uniform ball."""
    n, R, w = 4096, 10e-6, 50.0
    pos = wl.uniform_sphere(n, R, seed=13)
    K = KE2_M * n * w / R ** 3
    t_unit = 1.0 / math.sqrt(2 * K)
    s_end = 2.0
    T = t_unit * (math.sqrt(s_end * (s_end - 1)) + math.log(math.sqrt(s_end) + math.sqrt(s_end - 1)))
    nsteps = 200
    eps = 1e-3 * R
    d0 = oracle.diagnostics(pos, np.zeros_like(pos), w)
    p, v, a = oracle.vv_run(pos, np.zeros_like(pos), None, w, eps, T / nsteps, nsteps)
    d1 = oracle.diagnostics(p, v, w)
    ratio = d1["rms_radius"] / d0["rms_radius"]
    assert abs(ratio / s_end - 1) < 0.02, ratio
    pmag = math.sqrt(d1["px"] ** 2 + d1["py"] ** 2 + d1["pz"] ** 2)
    c = oracle.constants()
    assert pmag < 1e-12 * c["me"] * w * np.linalg.norm(v, axis=1).sum()


# --- paper setup arithmetic and workload generators ---------------------------------------

def test_paper_setup_weights_and_spacing():
    g = json.load(open(os.path.join(GOLD, "paper_setup.json")))
    l16 = g["lattice_16"]
    w = wl.lattice_weight(l16["n0_per_m3"], l16["side_m"], l16["n_particles"])
    assert round(w, l16["w_printed_digits"]) == l16["w_printed"]
    assert abs(wl.PAPER_LATTICE.w - w) == 0.0 and wl.PAPER_LATTICE.dt == l16["dt_s"]
    l32 = g["lattice_32"]
    w32 = wl.lattice_weight(l16["n0_per_m3"], l16["side_m"], l32["n_particles"])
    assert round(w32, l32["w_printed_digits"]) == l32["w_printed"]
    sp = g["lattice_8_spacing"]
    lat = wl.cube_lattice(sp["n_side"], l16["side_m"])
    xs = np.unique(lat[:, 0])
    np.testing.assert_allclose(np.diff(xs), sp["spacing_m"], rtol=1e-12)
    assert [k ** 3 for k in g["np_sweep"]["n_side"]][0] == g["np_sweep"]["first"]
    assert [k ** 3 for k in g["np_sweep"]["n_side"]][-1] == g["np_sweep"]["last"]
