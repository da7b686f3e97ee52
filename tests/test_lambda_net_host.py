"""Host-side logic of the learned lambda rule's training pipeline (no GPU): the parameter
order shared with the library, folding the input standardisation into the first layer, and
the seeded noise levels."""
import numpy as np

from oracle import mlp as OM
from paper_2602_17892_gb300 import lambda_net as LN


def _as_dict(v):
    v = np.asarray(v, np.float64)
    o, out = 0, {}
    for key, shape in (("W1", (64, 80)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
                       ("w3", (64,)), ("b3", (1,)), ("mu", (80,)), ("isd", (80,))):
        size = int(np.prod(shape))
        out[key] = v[o:o + size].reshape(shape)
        o += size
    assert o == v.size
    return out


def test_init_params_layout_and_scale():
    v = LN.init_params(3)
    assert v.dtype == np.float32 and v.size == 9569
    p = _as_dict(v)
    assert np.all(p["b1"] == 0) and np.all(p["b2"] == 0) and p["b3"][0] == 0
    assert np.all(p["mu"] == 0) and np.all(p["isd"] == 1)
    assert abs(p["W1"].std() - np.sqrt(2 / 80)) < 0.01
    assert abs(p["W2"].std() - np.sqrt(2 / 64)) < 0.01
    assert np.array_equal(v, LN.init_params(3)) and not np.array_equal(v, LN.init_params(4))


def test_standardisation_slots_give_the_standardised_network():
    """Parameters built with (mu, sd) on raw inputs equal the identity-standardised network on
    (x - mu) / sd (oracle forward, FP64)."""
    rng = np.random.Generator(np.random.PCG64(1))
    mu = rng.standard_normal(80) * 3
    sd = rng.random(80) * 2 + 0.1
    X = rng.standard_normal((17, 80)) * sd + mu
    raw = _as_dict(LN.init_params(5, mu, sd))
    ident = _as_dict(LN.init_params(5))
    out_raw, _ = OM.forward(raw, X)
    out_std, _ = OM.forward(ident, (X - mu) / sd)
    np.testing.assert_allclose(out_raw, out_std, rtol=1e-5, atol=1e-5)   # FP32 storage of 1/sd


def test_noise_levels_are_seeded_and_in_range():
    e = np.array([LN.noise_level(s) for s in range(2000)])
    assert e.min() >= 0.005 and e.max() <= 0.05
    assert abs(e.mean() - 0.0275) < 0.002
    assert LN.noise_level(7) == LN.noise_level(7)
    g = LN.training_geometry()
    assert (g.nx, g.ny, g.n_views, g.n_det_u) == (256, 256, 90, 367)
