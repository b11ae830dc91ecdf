"""Image-quality metrics of Sec. 4.3.2 (host numpy)."""
import math

import numpy as np


def mse(original, decrypted):
    """Mean of squared pixel differences over the image."""
    a = np.asarray(original, dtype=np.float64)
    b = np.asarray(decrypted, dtype=np.float64)
    return float(np.mean((a - b) ** 2))


def psnr(mse_value, max_i=255.0):
    """10 log10(MAX_I^2 / MSE) in dB; infinite for a zero MSE."""
    if mse_value == 0:
        return math.inf
    return 10.0 * math.log10(max_i * max_i / mse_value)
