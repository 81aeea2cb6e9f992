"""Pin of the oracle's network gradient (plain FP64 model) against central
finite differences, through the output mapping (scale exp, quaternion
increment, opacity logit, normal of R(q))."""
import numpy as np

import oracle.mlp as om


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    n = 7
    p = om.init_params(1)
    p["W4"] = rng.standard_normal((om.OUT_PAD, om.HID)) * 0.05
    p["W4"][om.OUT:] = 0
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    p["b4"] = np.zeros(om.OUT_PAD)
    p["b4"][:om.OUT] = rng.standard_normal(om.OUT) * 0.1
    x = rng.standard_normal((n, om.IN))
    s0 = rng.uniform(0.5, 2.0, (n, 3))
    q0 = rng.standard_normal((n, 4))
    o0 = np.full(n, 0.9)
    up = dict(scale=rng.standard_normal((n, 3)), quat=rng.standard_normal((n, 4)),
              opacity=rng.standard_normal(n), normal=rng.standard_normal((n, 3)))
    g = om.loss_grad_params(p, x, s0, q0, o0, up, rounding=False)
    worst = 0.0
    for k in ("W1", "W2", "W3", "W4", "b1", "b2", "b3", "b4"):
        flat = p[k].reshape(-1)
        picks = rng.choice(flat.size, size=min(25, flat.size), replace=False)
        if k in ("W4", "b4"):
            picks = [i for i in picks if (i // (om.HID if k == "W4" else 1)) < om.OUT]
        for i in picks:
            h = 1e-6 * max(1.0, abs(flat[i]))
            old = flat[i]
            flat[i] = old + h
            lp = om.linear_outputs(p, x, s0, q0, o0, up)
            flat[i] = old - h
            lm = om.linear_outputs(p, x, s0, q0, o0, up)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[i]
            err = abs(fd - an) / max(1.0, abs(fd))
            worst = max(worst, err)
            assert err < 1e-6, (k, i, fd, an)
    assert worst < 1e-6
