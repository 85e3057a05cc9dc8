"""CPU checks of the seeded input generators against the workload definitions
they implement (the generators hold no arithmetic of the method itself)."""
import numpy as np

from paper_1104_5330_gb300 import inputs as I


def test_shell_scattering_has_the_stated_optical_depth():
    """Lambert-shell plasma: largest at R1, zero at R2, and int kappa_s dr = tau
    along a radial line where the 0.1 modulation vanishes (theta = pi/2)."""
    x, w = np.polynomial.legendre.leggauss(40)
    R1, R2, tau = 0.5, 1.0, 5.0
    r = 0.5 * (R1 + R2) + 0.5 * (R2 - R1) * x
    ks = I.shell_scattering(r, np.array([np.pi / 2]), np.array([0.3]), R1, R2, tau)[0, :, 0, 0]
    assert abs(0.5 * (R2 - R1) * np.dot(w, ks) - tau) < 1e-12
    edge = I.shell_scattering(np.array([R1, R2]), np.array([1.0]), np.array([0.4]), R1, R2, tau)
    assert edge[0, 1, 0, 0] == 0.0 and edge[0, 0, 0, 0] > 0.0


def test_lambert_inflow_is_cosine_on_outgoing_directions():
    NT = 8
    Th = np.pi * (np.arange(NT) + 0.5) / NT
    g1, g2 = I.lambert_inflow(Th, 3, 4, 6, groups=2, F0=2.0)
    assert g1.shape == (2, 3, 4, NT // 2, 6) and np.all(g2 == 0)
    assert np.allclose(g1[1, 2, 3, :, 5], 2.0 * np.cos(Th[:NT // 2]))
    assert np.all(np.cos(Th[:NT // 2]) > 0)


def test_nucleon_densities_are_positive_with_a_bounded_proton_fraction():
    r, th, ph = np.linspace(0.2, 1, 7), np.linspace(0.1, 3.0, 5), np.linspace(0, 6, 6)
    An, Ap = I.nucleon_densities(r, th, ph, 3, 1104, 0.2, 1.0)
    assert An.shape == (3, 7, 5, 6) and np.all(An > 0) and np.all(Ap > 0)
    yp = Ap / (An + Ap)
    assert 0.05 < yp.min() and yp.max() < 0.51


def test_signed_field_covers_minus_one_to_one():
    f = I.signed_field(np.linspace(0.2, 1, 9), np.linspace(0.1, 3, 6), np.linspace(0, 6, 8),
                       2, 7, 0.2, 1.0)
    for g in range(2):
        assert abs(f[g].min() + 1) < 1e-15 and abs(f[g].max() - 1) < 1e-15
