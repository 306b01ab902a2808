"""Pins for the oracle's EM readings: Fresnel coefficients with the ITU-R
P.2040 complex permittivity, their derivatives, free-space LOS amplitude and
delay.  Each check uses an expression or a property independent of the
oracle's own formula (textbook special cases, Snell-form coefficients,
complex-step derivatives, reciprocity).  CPU only."""
import cmath

import numpy as np
import pytest

import oracle

C0 = 299792458.0
EPS0 = 8.8541878128e-12
F = 28e9


def eta_of(eps_r, sigma, f=F):
    return complex(eps_r, -sigma / (2 * np.pi * f * EPS0))


@pytest.mark.parametrize("eps_r,sigma", [(5.3, 0.03), (3.0, 0.01), (2.0, 0.1), (7.0, 0.001)])
def test_normal_incidence(eps_r, sigma):
    eta = eta_of(eps_r, sigma)
    ref = (1 - cmath.sqrt(eta)) / (1 + cmath.sqrt(eta))
    for pol in (0, 1):
        g = oracle.fresnel(eps_r, sigma, F, 1.0, pol)
        # TM sign convention (eta cos - s)/(eta cos + s) is the negative of TE at normal incidence
        want = ref if pol == 0 else -ref
        assert abs(g - want) < 1e-14


def test_grazing_tends_to_minus_one():
    for pol in (0, 1):
        g = oracle.fresnel(5.3, 0.03, F, 1e-9, pol)
        assert abs(g + 1) < 1e-6


def test_brewster_zero_lossless_tm():
    for eps_r in (2.0, 3.0, 5.3, 7.0):
        tb = np.arctan(np.sqrt(eps_r))
        g = oracle.fresnel(eps_r, 0.0, F, np.cos(tb), 1)
        assert abs(g) < 1e-14
        assert abs(oracle.fresnel(eps_r, 0.0, F, np.cos(tb), 0)) > 0.1


def test_lossy_magnitude_below_one_and_snell_form():
    rng = np.random.default_rng(0)
    for _ in range(200):
        eps_r, sigma = rng.uniform(1.5, 8), 10 ** rng.uniform(-3, -1)
        c = rng.uniform(1e-3, 1.0)
        eta = eta_of(eps_r, sigma)
        # Snell form: n2 = sqrt(eta), cos theta_t = sqrt(1 - sin^2 / eta)
        n2 = cmath.sqrt(eta)
        ct = cmath.sqrt(1 - (1 - c * c) / eta)
        te = (c - n2 * ct) / (c + n2 * ct)
        tm = (n2 * c - ct) / (n2 * c + ct)
        g0 = oracle.fresnel(eps_r, sigma, F, c, 0)
        g1 = oracle.fresnel(eps_r, sigma, F, c, 1)
        assert abs(g0) < 1 and abs(g1) < 1
        assert abs(g0 - te) < 1e-12
        assert abs(g1 - tm) < 1e-12


def test_fresnel_derivative_complex_step():
    """dGamma/deta against a central difference along the real axis and
    along the imaginary axis (holomorphy)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        eta = complex(rng.uniform(1.5, 8), -rng.uniform(1e-3, 0.1))
        c = rng.uniform(0.05, 1.0)
        for pol in (0, 1):
            d = oracle.dfresnel_deta(eta, c, pol)
            h = 1e-6
            fr = (oracle.fresnel_eta(eta + h, c, pol) - oracle.fresnel_eta(eta - h, c, pol)) / (2 * h)
            fi = (oracle.fresnel_eta(eta + 1j * h, c, pol) - oracle.fresnel_eta(eta - 1j * h, c, pol)) / (2j * h)
            assert abs(d - fr) < 1e-7 * max(1, abs(d))
            assert abs(d - fi) < 1e-7 * max(1, abs(d))


def test_los_amplitude_and_delay(room):
    """Empty scene region: LOS path a = lambda/(4 pi d), tau = d/c for
    TX (1,1,1.5) -> RX (4,3,1.2), d = sqrt(13.09) m."""
    sc = oracle.OracleScene(room.pos, room.nrm, room.surf, room.mat, r_p=0.05)
    p = oracle.SimParams(max_depth=1, capture=0, n_rays=16, r_rx=0.1)
    sim = oracle.OracleSim(sc, room.tx, room.rx, p)
    P = sim.paths()
    los = np.nonzero(P["k"] == 0)[0]
    assert los.size == 1
    d = np.sqrt(13.09)
    lam = C0 / F
    a, _ = sim.field(room.eps_r, room.sigma, room.scat)
    # tx and rx are float32 inputs; d from them
    d32 = np.linalg.norm(room.rx[0].astype(np.float64) - room.tx.astype(np.float64))
    assert abs(a[los[0]] - lam / (4 * np.pi * d32)) < 1e-14 * lam / (4 * np.pi * d32)
    assert abs(a[los[0]] - lam / (4 * np.pi * d)) < 1e-7 * lam / (4 * np.pi * d)
    assert P["tau"][los[0]] == pytest.approx(d32 / C0, rel=1e-14)
    assert d32 == pytest.approx(d, rel=1e-7)


def test_diffuse_power_off_a_plane_is_the_lambertian_integral():
    """The diffuse reading gives a scatter cell of area rho^2 the amplitude
    lambda/(4 pi) sqrt(rho^2 cos_i cos_s / pi) / (r_i r_s), i.e. a Lambertian
    lobe.  Summed over a flat plane, the powers |a|^2 / (lambda/4 pi)^2
    are then a midpoint Riemann sum of the radiometric integral
    int x_t x_r / (pi r_i^3 r_s^3) dA over a wall x = 0 (a vertical plane, so
    that the incidence cosine is not a z component).  One ray per DPS (the DPS-directed
    launch) scatters at each DPS's reception point: with four points per
    voxel axis these are the centres of rho-sized cells, so the sum must meet
    a fine quadrature of the integral over those cells to the midpoint
    rule's O(rho^2) error."""
    rho = 0.0625
    g = -1.5 + np.arange(48 * 4) * (rho / 4)  # 48 voxels, 4 points per axis in each
    X, Y = np.meshgrid(g, g, indexing="ij")
    pos = np.column_stack([np.zeros(X.size), X.ravel(), Y.ravel()]).astype(np.float32)
    nrm = np.tile(np.array([1, 0, 0], np.float32), (pos.shape[0], 1))
    n = pos.shape[0]
    osc = oracle.OracleScene(pos, nrm, np.zeros(n, np.uint16), np.zeros(n, np.uint8), rho=rho,
                             r_p=0.05, grid_cell=0.25)
    tx = np.array([1.0, 0.3, -0.2])
    rx = np.array([[0.8, -0.4, 0.5]])
    sim = oracle.OracleSim(osc, tx, rx, oracle.SimParams(max_depth=1, capture=1, diffuse=1,
                                                         n_rays=0, launch=1))
    P = sim.paths()
    dif = P["type"] == 1
    assert dif.sum() == osc.n_dps == 48 * 48
    lam = C0 / F
    got = np.sum(P["geo"][dif] ** 2) / (lam / (4 * np.pi)) ** 2
    # the cells: voxels start at the first point; the reception point sits
    # 1.5 point spacings into each voxel, so the cells centred there start
    # rho/8 before it
    x0 = -1.5 + 1.5 * rho / 4 - rho / 2
    M = 4000
    xs = x0 + (np.arange(M) + 0.5) * (48 * rho / M)
    XX, YY = np.meshgrid(xs, xs, indexing="ij")
    ri2 = tx[0] ** 2 + (XX - tx[1]) ** 2 + (YY - tx[2]) ** 2
    rs2 = rx[0, 0] ** 2 + (XX - rx[0, 1]) ** 2 + (YY - rx[0, 2]) ** 2
    want = np.sum(tx[0] * rx[0, 0] / (np.pi * ri2 ** 1.5 * rs2 ** 1.5)) * (48 * rho / M) ** 2
    assert got == pytest.approx(want, rel=1e-3)
