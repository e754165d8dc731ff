"""Pins of the oracle's condensed-history transport against closed forms.

* CSDA: with straggling, scattering and nuclear removal off, every proton
  stops at the integrated-stopping-power range (to 0.1 mm, here 0.02 mm),
  in water, in a denser medium (range / SPR) and through slabs (sum of
  water-equivalent thicknesses).
* R80 of the full-physics depth-dose within 0.5 mm of the CSDA range.
* Lateral spread of a zero-width pencil within 5 % of Fermi-Eyges theory
  with the Highland scattering power, integrated independently here.
* Primary fluence within 1 % of exp(-integral of Sigma) up to 0.9 R.
* Energy balance: deposited + escaped + removed = incident.
* Symmetry and exact additivity over history ranges.
"""
import math

import numpy as np
import pytest

from paper_1809_03927_gb300 import workloads as W

X0_MM = 360.8


def _r80(depth_dose, bin_mm):
    dd = depth_dose
    k = int(np.argmax(dd))
    m = dd[k]
    kk = k + int(np.argmax(dd[k:] < 0.8 * m))
    z = (np.arange(dd.shape[0]) + 0.5) * bin_mm
    return z[kk - 1] + (z[kk] - z[kk - 1]) * (dd[kk - 1] - 0.8 * m) / (dd[kk - 1] - dd[kk])


@pytest.mark.parametrize("energy", [70.0, 150.0, 200.0])
def test_csda_range_water(orc, energy):
    ph = W.water_phantom()
    pl = W.pencil_plan(energy=energy, sigma=0.0)
    r = orc.transport(ph, pl, 64, 1, physics=0)
    assert r["end_weight"] > 0
    assert abs(r["end_depth"] - orc.range_mm(energy)) < 0.02


def test_csda_range_scales_with_spr(orc):
    """Uniform bone-like medium (HU 1200): the range is R_w / SPR; an extra
    stopping-power scale s shortens it to R_w / (s SPR)."""
    ph = W.water_phantom(hu=1200)
    pl = W.pencil_plan(energy=150.0, sigma=0.0)
    spr = orc.spr(1200)
    r = orc.transport(ph, pl, 16, 1, physics=0)
    assert abs(r["end_depth"] - orc.range_mm(150.0) / spr) < 0.02
    r = orc.transport(ph, pl, 16, 1, physics=0, spr_scale=1.035)
    assert abs(r["end_depth"] - orc.range_mm(150.0) / (1.035 * spr)) < 0.02


def test_csda_range_through_slabs(orc):
    """Water 20 mm, lung 40 mm, bone 10 mm: stopping depth = 70 mm + (R_w -
    water-equivalent thickness of the slabs)."""
    ph = W.slab_phantom(n=128)
    pl = W.pencil_plan(energy=150.0, sigma=0.0)
    wet = 20.0 * orc.spr(0) + 40.0 * orc.spr(-740) + 10.0 * orc.spr(1200)
    want = 70.0 + (orc.range_mm(150.0) - wet)
    r = orc.transport(ph, pl, 16, 1, physics=0)
    assert abs(r["end_depth"] - want) < 0.02


def test_straggling_keeps_mean_range(orc):
    ph = W.water_phantom()
    pl = W.pencil_plan(energy=150.0, sigma=0.0)
    r = orc.transport(ph, pl, 4000, 3, physics=orc.PHYS_STRAGGLING)
    assert abs(r["end_depth"] - orc.range_mm(150.0)) < 0.1


def _bohr_range_sd(orc, e0):
    """Range straggling of the Bohr model, integrated here independently of
    the transport: sigma_R^2 = int k(E) / S(E)^3 dE from the cut-off to E0,
    with k the Bohr variance per mm of water and S the stopping power in
    MeV/mm (each energy-loss fluctuation dE shifts the range by dE / S)."""
    integrate = pytest.importorskip("scipy.integrate")
    v, _ = integrate.quad(lambda e: orc.bohr_var(e, 1.0) / (orc.bethe_sw(e) / 10.0) ** 3,
                          0.5, e0, limit=400, epsrel=1e-10)
    return math.sqrt(v)


def _line_phantom(dz, depth_mm):
    """One column of water voxels dz long along +z, 100 mm wide laterally,
    so a zero-width pencil without scattering crosses only z faces."""
    nz = int(math.ceil(depth_mm / dz))
    return W.Phantom(np.zeros((nz, 1, 1), np.int16), (100.0, 100.0, dz), (-50.0, -50.0, 0.0))


@pytest.mark.parametrize("energy,dz,n,tol", [(150.0, 0.05, 10000, 0.025), (70.0, 0.1, 20000, 0.02),
                                             (150.0, 0.5, 20000, 0.02), (150.0, 2.0, 20000, 0.03),
                                             (70.0, 2.0, 20000, 0.035)])
def test_range_straggling_matches_bohr(orc, energy, dz, n, tol):
    """With straggling alone, the standard deviation of the stopping depth of
    a zero-width pencil is the Bohr range straggling (about 1.1 % of the
    range), on voxels of 0.05 to 2 mm, i.e. for steps from 0.05 mm to 2 mm:
    the loss model keeps the step's mean and variance whatever its length.
    The coarse grids sit up to 2 % low (the discretisation of the
    condensed-history steps, independent of the loss distribution); a
    Gaussian fluctuation truncated at +-mean loss gives 0.88 at 0.05 mm and
    150 MeV and fails.  Statistical error of the sd: 1/sqrt(2n), 0.5-0.7 %."""
    want = _bohr_range_sd(orc, energy)
    ph = _line_phantom(dz, orc.range_mm(energy) + 20.0)
    r = orc.transport(ph, W.pencil_plan(energy=energy, sigma=0.0), n, 11,
                      physics=orc.PHYS_STRAGGLING, max_steps=100000)
    assert r["end_weight"] == n
    assert abs(r["end_depth_sd"] / want - 1.0) < tol, (r["end_depth_sd"], want)
    assert abs(r["end_depth"] - orc.range_mm(energy)) < 0.05


@pytest.mark.parametrize("energy", [70.0, 150.0])
def test_r80_full_physics(orc, energy):
    ph = W.water_phantom(nx=32, ny=32)
    pl = W.pencil_plan(energy=energy, sigma=0.0)
    bin_mm = 0.1
    r = orc.transport(ph, pl, 20000, 5, depth_bin_mm=bin_mm, n_depth_bins=3200)
    assert abs(_r80(r["depth_dose"], bin_mm) - orc.range_mm(energy)) < 0.5


def _fermi_eyges_sigma(orc, energy, depths, hu=0):
    """sigma^2(z) = int_0^z (z - z')^2 T(z') dz', T = d theta0^2 / dz with the
    Highland scattering power of the cumulative form (thickness u = z rho/X0)
    along the CSDA energy E(z) = E_w(R_w - z SPR) in a uniform medium."""
    integrate = pytest.importorskip("scipy.integrate")
    r0 = orc.range_mm(energy)
    rho, spr = orc.rho(hu), orc.spr(hu)
    b = 0.038

    def t_of(zp):
        u = zp * rho / X0_MM
        if u <= 0.0:
            return 0.0
        e = orc.energy_from_range(r0 - zp * spr)
        lu = math.log(u)
        dg = (1 + b * lu) ** 2 + 2 * b * (1 + b * lu)
        return (13.6 / orc.pv(e)) ** 2 * dg * rho / X0_MM

    out = []
    for z in depths:
        v, _ = integrate.quad(lambda zp: (z - zp) ** 2 * t_of(zp), 0.0, z, limit=400,
                              points=[1e-6, 1e-3, 1.0])
        out.append(math.sqrt(v))
    return np.array(out)


@pytest.mark.parametrize("hu", [0, 1200, -740])
def test_lateral_sigma_fermi_eyges(orc, hu):
    """Zero-width pencil in water, in bone-like and in lung-like media."""
    energy = 150.0 if hu != -740 else 70.0
    ph = W.water_phantom(nx=64, ny=64, nz=100 if hu != -740 else 128, hu=hu)
    pl = W.pencil_plan(energy=energy, sigma=0.0)
    n = 20000
    r0 = orc.range_mm(energy) / orc.spr(hu)
    r = orc.transport(ph, pl, n, 9, plane_mm=1.0, n_planes=int(r0) + 2)
    ks = [int(f * r0) - 1 for f in (0.2, 0.4, 0.6, 0.8, 0.9)]
    w = r["plane_w"][ks]
    m1 = r["plane_m1"][:, ks] / w
    m2 = r["plane_m2"][:, ks] / w
    sig = np.sqrt(m2 - m1 ** 2)
    fe = _fermi_eyges_sigma(orc, energy, [k + 1.0 for k in ks], hu)
    for axis in range(2):
        rel = np.abs(sig[axis] - fe) / fe
        assert np.all(rel < 0.05), (sig[axis], fe)


def _survival(orc, energy, z):
    integrate = pytest.importorskip("scipy.integrate")
    r0 = orc.range_mm(energy)
    v, _ = integrate.quad(lambda zp: orc.sigma_nuc(orc.energy_from_range(r0 - zp)) / 10.0, 0.0, z,
                          limit=200)
    return math.exp(-v)


@pytest.mark.parametrize("physics", ["nuclear", "all"])
def test_primary_fluence(orc, physics):
    energy = 150.0
    ph = W.water_phantom(nx=64, ny=64, nz=100)
    pl = W.pencil_plan(energy=energy, sigma=0.0)
    n = 20000
    phys = orc.PHYS_NUCLEAR if physics == "nuclear" else orc.PHYS_ALL
    r = orc.transport(ph, pl, n, 13, physics=phys, plane_mm=1.0, n_planes=190)
    r0 = orc.range_mm(energy)
    for f in (0.1, 0.3, 0.5, 0.7, 0.9):
        k = int(f * r0) - 1
        want = _survival(orc, energy, k + 1.0)
        got = r["plane_w"][k] / n
        assert abs(got - want) / want < 0.01, (f, got, want)


def test_energy_balance(orc):
    ph = W.slab_phantom(n=64)
    pl = W.slab_plan(n_layers=3, nx=3, ny=2)
    r = orc.transport(ph, pl, 3000, 21)
    dep, esc, rem, inc = r["ledger"]
    assert abs(dep + esc + rem - inc) <= 1e-9 * inc
    assert abs(r["edep"].sum() - dep) <= 1e-9 * inc
    assert esc > 0 and rem > 0


def test_lateral_escape_at_birth(orc):
    ph = W.water_phantom(nx=16, ny=16, nz=16)
    pl = W.pencil_plan(energy=100.0, sigma=0.0, x=500.0)
    r = orc.transport(ph, pl, 100, 1)
    dep, esc, rem, inc = r["ledger"]
    assert dep == 0.0 and rem == 0.0 and esc == inc


def test_history_ranges_add_up(orc):
    ph = W.water_phantom(nx=32, ny=32, nz=100)
    pl = W.pencil_plan(energy=120.0)
    n = 2000
    a = orc.transport(ph, pl, n, 4, hist_range=(0, 700), nthreads=1)
    b = orc.transport(ph, pl, n, 4, hist_range=(700, n), nthreads=3)
    c = orc.transport(ph, pl, n, 4, nthreads=2)
    np.testing.assert_allclose(a["edep"] + b["edep"], c["edep"], rtol=1e-12, atol=1e-9)
    assert a["steps"] + b["steps"] == c["steps"]


def test_beam_direction_symmetry(orc):
    """A beam along -z through the same water phantom gives the mirrored
    depth-dose; beams along +x and +y through transposed phantoms give the
    same depth-dose (statistically: different transverse frames)."""
    n = 6000
    ph = W.water_phantom(nx=32, ny=32, nz=100)
    pl = W.pencil_plan(energy=120.0)
    ref = orc.transport(ph, pl, n, 7)["edep"].sum(axis=(1, 2))
    mir = W.Phantom(ph.hu, ph.d, ph.origin, 2, -1)
    got = orc.transport(mir, pl, n, 7)["edep"].sum(axis=(1, 2))[::-1]
    hx = np.ascontiguousarray(np.transpose(ph.hu, (2, 1, 0)))          # beam axis -> x
    phx = W.Phantom(hx, ph.d, (0.0, -32.0, -32.0), 0, 1)
    gx = orc.transport(phx, pl, n, 7)["edep"].sum(axis=(0, 1))
    hy = np.ascontiguousarray(np.transpose(ph.hu, (1, 0, 2)))          # beam axis -> y
    phy = W.Phantom(hy, ph.d, (-32.0, 0.0, -32.0), 1, 1)
    gy = orc.transport(phy, pl, n, 7)["edep"].sum(axis=(0, 2))
    peak = ref.max()
    for g in (got, gx, gy):
        assert np.max(np.abs(g - ref)) < 0.03 * peak
        assert abs(g.sum() - ref.sum()) < 0.01 * ref.sum()


def test_normalise_unit_conversion(orc):
    """1 MeV in 1 cm^3 of unit-density medium with one proton per history is
    1.602176634e-13 J / 1e-3 kg = 1.602176634e-10 Gy."""
    d = orc.normalise(np.array([1.0, 2.0]), np.array([1.0, 2.0]), 1.0, 1.0)
    np.testing.assert_allclose(d, [1.602176634e-10, 1.602176634e-10], rtol=1e-15)
    d = orc.normalise(np.array([3.0]), np.array([1.0]), 1e6, 0.008)
    np.testing.assert_allclose(d, [3.0 * 1e6 * 1.602176634e-13 / 8e-6], rtol=1e-15)
