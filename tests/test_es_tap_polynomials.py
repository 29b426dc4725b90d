"""Why the spreader evaluates its ES taps with sqrt + exp2 rather than with
polynomials on the FMA pipe: FP64 Chebyshev fits of each tap of the w = 7,
beta = 2.30 w kernel as a function of the sample's fractional offset.

The ES kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) (Barnett, Magland and
af Klinteberg 2019) is smooth inside its support, so a tap whose window stays
inside it fits a low-degree polynomial well; but sqrt(1 - z^2) has a branch
point at |z| = 1, so the two edge taps, whose windows end there, converge
slowly.  The degrees found here set the FMA cost a polynomial tap would have
(one FMA per degree per tap per sample).  CPU only; no library code."""
import numpy as np

W = 7
BETA = 2.30 * W


def _tap_values(t, u):
    """Tap t (0..W-1) of a sample whose first tap sits a fraction u in [0, 1]
    of a cell past the kernel's left end, normalised to the kernel's peak."""
    z = -1.0 + (2.0 / W) * (u + t)
    return np.exp(BETA * (np.sqrt(np.maximum(1.0 - z * z, 0.0)) - 1.0))


def _fit_error(t, degree, u):
    x = 2.0 * u - 1.0
    f = _tap_values(t, u)
    c = np.polynomial.chebyshev.chebfit(x, f, degree)
    return np.max(np.abs(np.polynomial.chebyshev.chebval(x, c) - f))


def test_inner_taps_need_degree_eight():
    u = np.linspace(0.0, 1.0, 20001)
    for t in range(1, W - 1):
        assert _fit_error(t, 8, u) < 5e-9, t
        assert _fit_error(t, 6, u) > 5e-9, t


def test_edge_taps_converge_slowly():
    u = np.linspace(0.0, 1.0, 20001)
    for t in (0, W - 1):
        errs = [_fit_error(t, d, u) for d in (8, 10, 12)]
        assert all(e > 3e-8 for e in errs), (t, errs)
        # each two degrees buy less than a factor 1.3: the branch point at |z| = 1
        assert errs[0] / errs[2] < 1.6, (t, errs)


def test_taps_are_mirror_images():
    u = np.linspace(0.0, 1.0, 101)
    for t in range(W):
        assert np.allclose(_tap_values(t, u), _tap_values(W - 1 - t, 1.0 - u), rtol=1e-12, atol=0)
