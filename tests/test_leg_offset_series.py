"""The series the snapshot phase-word kernel uses for an antenna's leg offset (Sec. II-E, Eq. 7),
checked on the CPU against the exact difference of two lengths.

An antenna at x_ref + e sees a hit at u from the reference antenna (s = |u|) at a length
differing by |u - e| - s = s (sqrt(1 + x) - 1), x = (|e|^2 - 2 u.e) / s^2.  The kernel takes
num / (2 s) (1 - x/4 + x^2/8 - 5 x^3/64 + 7 x^4/128) for |x| <= 1/20 and the rationalised
form num / (|u - e| + s) beyond; the truncation must stay below FP32 resolution there."""
import numpy as np

X_MAX = 0.05


def series(num, s):
    x = num / (s * s)
    p = 1.0 + x * (-0.25 + x * (1.0 / 8.0 + x * (-5.0 / 64.0 + x * (7.0 / 128.0))))
    return num / (2.0 * s) * p


def test_series_truncation_below_fp32_resolution():
    x = np.concatenate([np.linspace(-X_MAX, X_MAX, 400001), [-X_MAX, X_MAX]])
    x = x[x != 0.0]
    s = 1.0
    exact = s * x / (np.sqrt(1.0 + x) + 1.0)   # s (sqrt(1 + x) - 1) without cancellation
    rel = np.abs(series(x * s * s, s) - exact) / np.abs(exact)
    assert rel.max() <= 1.4e-8            # below 2^-24 = 6e-8, the FP32 rounding of the result
    assert rel.max() >= 1.0e-8            # and the bound is not loose: x^5 term 21/512 x^5


def test_series_against_lengths_of_a_compact_array():
    """Random hits 3 to 150 m away, antenna offsets up to 2 cm: |x| stays far inside 1/20 and
    the series gives the length difference to a few 1e-12 m (FP64 here; the kernel's FP32
    arithmetic adds its own ~2^-23 of the offset)."""
    rng = np.random.default_rng(7)
    n = 20000
    r = rng.uniform(3.0, 150.0, n)
    d = rng.normal(size=(n, 3))
    u = d / np.linalg.norm(d, axis=1, keepdims=True) * r[:, None]
    e = rng.uniform(-0.02, 0.02, (n, 3))
    s = np.linalg.norm(u, axis=1)
    num = np.einsum("ij,ij->i", e, e) - 2.0 * np.einsum("ij,ij->i", u, e)
    x = num / (s * s)
    assert np.abs(x).max() < 0.02
    exact = np.linalg.norm(u - e, axis=1) - s
    assert np.abs(series(num, s) - exact).max() <= 5e-12


def test_rationalised_form_beyond_the_series_range():
    """Where |x| > 1/20 (antennas far apart, a near hit) the kernel keeps the rationalised form,
    which has no truncation: it equals the difference of lengths to rounding."""
    u = np.array([[0.5, 0.2, 0.1], [1.0, -0.3, 0.0]])
    e = np.array([[0.2, 0.0, 0.0], [0.0, 0.4, 0.1]])
    s = np.linalg.norm(u, axis=1)
    num = np.einsum("ij,ij->i", e, e) - 2.0 * np.einsum("ij,ij->i", u, e)
    assert (np.abs(num / (s * s)) > X_MAX).all()
    rationalised = num / (np.sqrt(s * s + num) + s)
    assert np.allclose(rationalised, np.linalg.norm(u - e, axis=1) - s, rtol=1e-12, atol=0.0)
