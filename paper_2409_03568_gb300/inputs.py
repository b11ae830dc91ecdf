"""Seeded synthetic inputs shaped like the paper's image workloads.

The paper evaluates on USC-SIPI images (Sec. 4.2), which are not available here. These
generators stand in for them: smooth random fields whose quantised histograms are skewed and
peaked, as natural images are, so frequent-value caching gets hits. Every generator is a pure
function of its seed. This module holds no cryptographic arithmetic; both the CUDA path's
tests/benchmarks and the CPU oracle's tests draw their inputs from it.
"""
import numpy as np

try:  # scipy is present on both the build host and the GPU hosts
    from scipy.ndimage import gaussian_filter as _gaussian_filter
except ImportError:  # pragma: no cover
    _gaussian_filter = None


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def _smooth(z, sigma):
    if _gaussian_filter is not None:
        return _gaussian_filter(z, sigma=sigma, mode="reflect")
    # separable Gaussian with reflect padding (fallback without scipy)
    r = int(4 * sigma + 0.5)
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    k /= k.sum()
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        zp = np.pad(z, pad, mode="symmetric")
        z = np.apply_along_axis(lambda v: np.convolve(v, k, mode="valid"), axis, zp)
    return z


def random_field_image(h, w, seed, channels=1, corr_px=6.0, mean=128.0, spread=48.0):
    """Gaussian random field (white N(0,1), Gaussian smoothing with the given correlation
    length, normalised to zero mean / unit variance) quantised as clip(round(mean + spread*z)).
    Returns uint8 [h, w] for one channel, [h, w, channels] otherwise (channels drawn
    independently from one seeded stream)."""
    rng = _rng(seed)
    planes = []
    for _ in range(channels):
        z = rng.standard_normal((h, w))
        z = _smooth(z, corr_px)
        z = (z - z.mean()) / max(z.std(), 1e-12)
        planes.append(np.clip(np.round(mean + spread * z), 0, 255).astype(np.uint8))
    return planes[0] if channels == 1 else np.stack(planes, axis=-1)


def uniform_image(h, w, seed, channels=1):
    """uint8 pixels uniform on 0..255."""
    shape = (h, w) if channels == 1 else (h, w, channels)
    return _rng(seed).integers(0, 256, size=shape, dtype=np.uint8)


def brightness_beta(seed, lo=-40.0, hi=40.0):
    """One brightness offset, uniform on [lo, hi]."""
    return float(_rng(seed).uniform(lo, hi))


def binary_pattern(h, w, seed, on=255):
    """Bernoulli(1/2) watermark pattern with values 0 / `on`."""
    return (_rng(seed).integers(0, 2, size=(h, w), dtype=np.uint8) * np.uint8(on)).astype(np.uint8)


def noisy_copy(img, seed, sigma_px=5.0):
    """clip(round(img + N(0, sigma^2))) -- the second image for matching."""
    rng = _rng(seed)
    noisy = np.asarray(img, dtype=np.float64) + rng.normal(0.0, sigma_px, size=np.shape(img))
    return np.clip(np.round(noisy), 0, 255).astype(np.uint8)


def ragged_batch(n_images, seed, side_lo=16, side_hi=128):
    """Square grayscale random-field images with sides uniform on [side_lo, side_hi]."""
    rng = _rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=n_images)
    return [random_field_image(int(s), int(s), seed=int(seed) * 1000 + i) for i, s in enumerate(sides)]
