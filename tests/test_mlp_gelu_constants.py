"""The tensor-core network evaluates GELU(z) = z Phi(z) with the Abramowitz &
Stegun 7.1.26 form of erf.  The constants are read from the CUDA source and the
formula is checked in FP64 against the error bound the handbook states
(|error| <= 1.5e-7) and against the normal CDF; a mistyped digit fails."""
import math
import re
from pathlib import Path

import numpy as np

SRC = Path(__file__).resolve().parents[1] / "paper_2404_02346_gb300" / "csrc" / "wlb_mlp.cu"


def _constants():
    text = SRC.read_text()
    out = {}
    for name in ("p", "a1", "a2", "a3", "a4", "a5"):
        m = re.search(r"kAS_%s = (-?[0-9.]+)f" % name, text)
        assert m, name
        out[name] = float(m.group(1))
    return out


def _erf_as(x, c):
    t = 1.0 / (1.0 + c["p"] * x)
    poly = t * (c["a1"] + t * (c["a2"] + t * (c["a3"] + t * (c["a4"] + t * c["a5"]))))
    return 1.0 - poly * np.exp(-x * x)


def test_erf_form_within_the_handbook_bound():
    c = _constants()
    x = np.linspace(0.0, 8.0, 200001)
    ref = np.array([math.erf(v) for v in x])
    assert np.abs(_erf_as(x, c) - ref).max() <= 1.5e-7


def test_gelu_from_the_form_matches_z_phi():
    from scipy.stats import norm
    c = _constants()
    z = np.linspace(-9.0, 9.0, 36001)
    x = np.abs(z) / math.sqrt(2.0)
    q = 0.5 * (1.0 - _erf_as(x, c))           # Phi(-|z|)
    g = 0.5 * z + np.abs(z) * (0.5 - q)       # z Phi(z) for either sign
    assert np.abs(g - z * norm.cdf(z)).max() <= 1.5e-7 * 9.0 / 2.0 + 1e-15
