"""Pins of the oracle's discrete elastic energy (the energy that the upwind-stability pin,
the library's energy reduction and its NaN/Inf sentinel are compared against).

E = sum_k int_k (rho |v|^2 / 2 + sigma : C^-1 sigma / 2). The compliance C^-1 is written
here independently, from Young's modulus and Poisson's ratio (eps_xx = (s_xx - nu (s_yy +
s_zz)) / E, eps_xy = (1 + nu) s_xy / E), and the energies are checked against closed forms:
a uniform state in a box of known volume, and exact P and S plane waves on the periodic unit
cube, whose kinetic and potential parts are equal (rho A^2 / 4 each for velocity amplitude A).
"""
import numpy as np
import pytest

from oracle import physics as ph
from oracle.mesh import Mesh
from oracle.scheme import Solver
from paper_2202_10313_gb300 import synth

RHO, VP, VS = 2700.0, 6000.0, 3464.0


def _young_poisson(lam, mu):
    return mu * (3 * lam + 2 * mu) / (lam + mu), lam / (2 * (lam + mu))


def _compliance_energy_ev(sig, lam, mu):
    """1/2 sigma : eps with eps from the engineering (E, nu) form of Hooke's law; Voigt
    (xx, yy, zz, xy, yz, xz), shear stresses counted twice in the double contraction."""
    E, nu = _young_poisson(lam, mu)
    sxx, syy, szz, sxy, syz, sxz = (sig[..., i] for i in range(6))
    exx = (sxx - nu * (syy + szz)) / E
    eyy = (syy - nu * (sxx + szz)) / E
    ezz = (szz - nu * (sxx + syy)) / E
    g = (1 + nu) / E
    return 0.5 * (sxx * exx + syy * eyy + szz * ezz + 2 * (sxy * g * sxy + syz * g * syz + sxz * g * sxz))


def test_compliance_density_matches_young_poisson_form():
    rng = np.random.default_rng(5)
    sig = rng.standard_normal((200, 6)) * 1e6
    lam = rng.uniform(0.2, 3.0, 200) * 1e10
    mu = rng.uniform(0.2, 3.0, 200) * 1e10
    got = ph.compliance_energy_density(sig, lam, mu)
    want = _compliance_energy_ev(sig, lam, mu)
    assert np.all(want > 0)
    assert np.abs(got / want - 1).max() < 1e-12


def test_compliance_of_pure_states():
    """Uniaxial stress s: s^2/(2E). Pure shear s_xy = t: t^2/(2 mu) (the double contraction
    counts the xy and yx components). Hydrostatic p: 3 p^2 / (2 (3 lam + 2 mu))."""
    lam, mu, s = 3.0e10, 2.0e10, 1.3e6
    E, _ = _young_poisson(lam, mu)
    uni = np.array([s, 0, 0, 0, 0, 0.0])
    shear = np.array([0, 0, 0, s, 0, 0.0])
    hyd = np.array([s, s, s, 0, 0, 0.0])
    assert abs(ph.compliance_energy_density(uni, lam, mu) / (s * s / (2 * E)) - 1) < 1e-14
    assert abs(ph.compliance_energy_density(shear, lam, mu) / (s * s / (2 * mu)) - 1) < 1e-14
    assert abs(ph.compliance_energy_density(hyd, lam, mu) / (3 * s * s / (2 * (3 * lam + 2 * mu))) - 1) < 1e-14


def test_uniform_state_energy_is_density_times_volume():
    """A constant state (projected exactly by any rule of degree >= 0) on a jittered graded
    box with layered material: E = sum over elements of vol_k (rho_k |v0|^2 / 2 + 1/2 s0 :
    C_k^-1 s0), with the element volumes from the vertex triple products and the box volume
    nx h x ny h x depth (boundary vertices move tangentially only)."""
    m = synth.graded_box(4, 3, 3, 200.0, 90.0, seed=4)
    mesh = Mesh(m["xyz"], m["tet"], m["face_bc"])
    mat = synth.layered(m, [150.0], [1300.0, 2600.0])
    s = Solver(4, 0, mesh, mat["rho"], mat["vp"], mat["vs"])
    s0 = np.array([2.0e6, -1.0e6, 0.5e6, 0.8e6, -0.3e6, 1.1e6])
    v0 = np.array([0.3, -0.2, 0.7])
    s.project(lambda x: np.tile(np.concatenate([s0, v0]), (len(x), 1)))
    x = m["xyz"][m["tet"]]
    vol = np.abs(np.einsum("ki,ki->k", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))) / 6
    assert abs(vol.sum() / (4 * 200.0 * 3 * 200.0 * m["depth"]) - 1) < 1e-12
    lam, mu = ph.lame(mat["rho"], mat["vp"], mat["vs"])
    dens = 0.5 * mat["rho"] * (v0 @ v0) + _compliance_energy_ev(s0[None, :], lam, mu)
    want = float(np.sum(vol * dens))
    assert abs(s.energy() / want - 1) < 1e-12


def _kinetic(s):
    return 0.5 * float(np.sum(s.mesh.detJ[:, None] * s.rho[:, None] * np.sum(s.Q[:, 6:9, :] ** 2, axis=1)))


@pytest.mark.parametrize("wave", ["P", "S"])
def test_plane_wave_energy_closed_form_and_equipartition(wave):
    """Exact plane wave of velocity amplitude 1 on the periodic unit cube, projected at
    order 5: kinetic and potential parts each equal rho/4 (int sin^2 = 1/2 over the cube),
    to the projection error. The analytic potential of the exact stress amplitude, from the
    (E, nu) compliance, is rho/2 per unit sin^2 as well."""
    kvec = 2 * np.pi * np.array([1.0, 1.0, 1.0])
    if wave == "P":
        fn = synth.p_plane_wave(RHO, VP, VS, kvec)
    else:
        fn = synth.s_plane_wave(RHO, VS, kvec, [1.0, -1.0, 0.0])
    r = fn(np.array([[1.0, 0.0, 0.0]]) / 12.0, 0.0)[0] / np.sin(kvec[0] / 12.0)   # amplitude vector
    lam, mu = ph.lame(RHO, VP, VS)
    assert abs(_compliance_energy_ev(r[:6], lam, mu) / (0.5 * RHO) - 1) < 1e-12
    assert abs(r[6:] @ r[6:] - 1) < 1e-12
    mm = synth.periodic_cube(4)
    mesh = Mesh(mm["xyz"], mm["tet"], mm["face_bc"], mm["period"])
    K = mesh.K
    s = Solver(5, 0, mesh, np.full(K, RHO), np.full(K, VP), np.full(K, VS))
    s.project(lambda x: fn(x, 0.0))
    e = s.energy()
    kin = _kinetic(s)
    pot = e - kin
    assert abs(kin / (RHO / 4) - 1) < 2e-3, kin
    assert abs(pot / (RHO / 4) - 1) < 2e-3, pot
    assert abs(pot / kin - 1) < 1e-3, (pot, kin)
