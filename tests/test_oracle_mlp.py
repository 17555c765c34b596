"""Pins of the oracle's learned-CDF model (monotone 1 -> 32 -> 32 -> 1 ReLU MLP)."""
import os
import types

import numpy as np
import pytest

from oracle import pgs_oracle as O
from paper_1611_00463_gb300 import inputs

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "pgs_oracle.py")


def random_raw(seed):
    g = np.random.default_rng(seed)
    raw = {"v1": g.normal(0, 0.5, 32), "b1": g.normal(0, 0.5, 32), "V2": g.normal(-1, 0.5, (32, 32)),
           "b2": g.normal(0, 0.3, 32), "v3": g.normal(-2, 0.5, 32), "b3": np.array(0.3)}
    raw["V2"] = np.where(O.mlp_block_mask(), raw["V2"], 0.0)
    return raw


def identity_weights():
    """y = x exactly: h1_0 = x, h2_0 = h1_0, y = h2_0 (products by 1 and sums with 0 are exact)."""
    eff = {"w1": np.zeros(32), "b1": np.zeros(32), "W2": np.zeros((32, 32)), "b2": np.zeros(32),
           "w3": np.zeros(32), "b3": np.array(0.0)}
    eff["w1"][0] = 1.0
    eff["W2"][0, 0] = 1.0
    eff["w3"][0] = 1.0
    return O.mlp_pack(eff)


def test_gradient_matches_finite_differences():
    for seed in range(3):
        raw = random_raw(seed)
        x = np.sort(np.random.default_rng(seed + 10).random(200))
        t = (np.arange(200) + 0.5) / 200
        _, g = O.mlp_loss_grad(raw, x, t)
        rng = np.random.default_rng(seed)
        for k in raw:
            flat = raw[k].reshape(-1)
            idx = range(flat.size) if flat.size <= 32 else rng.choice(flat.size, 24, replace=False)
            for i in idx:
                if k == "V2" and not O.mlp_block_mask().reshape(-1)[i]:
                    assert g[k].reshape(-1)[i] == 0.0
                    continue
                h = 1e-6
                plus = {kk: vv.copy() for kk, vv in raw.items()}
                minus = {kk: vv.copy() for kk, vv in raw.items()}
                plus[k].reshape(-1)[i] += h
                minus[k].reshape(-1)[i] -= h
                num = (O.mlp_loss_grad(plus, x, t)[0] - O.mlp_loss_grad(minus, x, t)[0]) / (2 * h)
                assert abs(num - g[k].reshape(-1)[i]) <= 1e-6 + 1e-4 * abs(num), (k, i)


def test_first_adam_step_is_lr_times_sign():
    # At step 1 the bias-corrected moments are m_hat = g and v_hat = g^2, so every
    # raw parameter moves by -lr g / (|g| + eps): about -lr sign(g).
    x = np.sort(inputs.exponential_u32(5000, 3).astype(np.float64)) / 2.0**32
    t = (np.arange(len(x)) + 0.5) / len(x)
    raw0 = O.mlp_init(x)
    _, g = O.mlp_loss_grad(raw0, x, t)
    raw1, _ = O.mlp_train(x, steps=1, lr=0.01)
    for k in raw0:
        want = raw0[k] - 0.01 * g[k] / (np.abs(g[k]) + 1e-8)
        if k == "V2":
            want = np.where(O.mlp_block_mask(), want, raw0[k])
        assert np.allclose(raw1[k], want, rtol=0, atol=1e-12), k


def test_init_knots_closed_form():
    x = np.arange(64, dtype=np.float64) / 64.0
    raw = O.mlp_init(x)
    q = x[[(2 * j + 1) * 64 // 32 for j in range(16)]]
    assert np.array_equal(raw["b1"][:16], -q) and np.array_equal(raw["b1"][16:], q)
    assert raw["V2"][3, 3] == 0.0 and raw["V2"][3, 4] == O.MLP_OFF_DIAG and raw["V2"][3, 20] == 0.0


def test_identity_network_buckets_are_integer_floor():
    w = identity_weights()
    for P in [1, 2, 7, 16, 1000, 1024]:
        # x = i / 4096 exactly in float32; bucket = min(P-1, floor(P i / 4096)).
        i = np.arange(0, 4097 + 300)
        x32 = (i.astype(np.float32) / np.float32(4096))
        got = O.mlp_bucket_f32(w, x32, P)
        want = np.minimum((P * i) // 4096, P - 1)
        assert np.array_equal(got, want), P


def test_effective_weights_are_monotone_and_forward_rises():
    for seed in range(5):
        eff = O.mlp_effective(random_raw(seed))
        w = O.mlp_pack(eff)
        assert O.mlp_monotone(w)
        x = np.linspace(-0.5, 1.5, 200_001)
        y, _ = O.mlp_forward64(eff, x)
        assert np.all(np.diff(y) >= -1e-12)
        b = O.mlp_bucket_f32(w, x.astype(np.float32), 257)
        assert np.all(np.diff(b) >= 0)


def test_halves_are_convex_and_concave():
    """The sign constraints make the +x half a rising convex function and the
    -x half a rising concave one (the model class is their sums): second
    differences on a uniform grid have the half's sign."""
    x = np.linspace(-0.5, 1.5, 20_001)
    half = np.arange(32) < 16
    for seed in range(5):
        eff = O.mlp_effective(random_raw(seed))
        for keep, sign in ((half, 1.0), (~half, -1.0)):
            e = dict(eff)
            e["w3"] = np.where(keep, eff["w3"], 0.0)
            e["b3"] = np.array(0.0)
            y, _ = O.mlp_forward64(e, x)
            assert np.all(np.diff(y) >= -1e-12)
            assert np.all(sign * np.diff(y, 2) >= -1e-12)


def test_float32_buckets_agree_with_float64_away_from_boundaries():
    eff = O.mlp_effective(random_raw(7))
    w = O.mlp_pack(eff)
    x = np.linspace(0, 1, 50_001).astype(np.float32)
    P = 64
    b32 = O.mlp_bucket_f32(w, x, P)
    y64, _ = O.mlp_forward64(O.mlp_unpack(w) | {}, x.astype(np.float64))
    p64 = P * np.clip(y64, 0, 1)
    far = np.abs(p64 - np.round(p64)) > 1e-3
    assert np.array_equal(b32[far], np.minimum(np.floor(p64[far]), P - 1).astype(np.int64))


def test_training_fits_a_smooth_cdf():
    x = np.sort(inputs.exponential_u32(8192, 3).astype(np.float64))
    x = (x - x[0]) / (x[-1] - x[0])
    t = (np.arange(len(x)) + 0.5) / len(x)
    raw0 = O.mlp_init(x)
    l0, _ = O.mlp_loss_grad(raw0, x, t)
    raw, l1 = O.mlp_train(x, steps=O.MLP_STEPS)
    assert l1 < 0.05 * l0 and l1 < 1e-3
    assert O.mlp_monotone(O.mlp_pack(O.mlp_effective(raw)))


def test_learned_buckets_semantics():
    keys = inputs.exponential_u32(20_000, 5)
    P = 16
    w = O.mlp_pack(O.mlp_effective(random_raw(3)))
    kmin, scale = O.mlp_norm(np.sort(keys))
    res = O.learned_buckets(keys, P, "u32", w, kmin, scale)
    e, cut = res["e"], res["cut"]
    assert e[0] == 0 and e[-1] == len(keys) and np.all(np.diff(e) >= 0)
    # Brute force: every key's bucket, counted per run.
    bounds = O.run_bounds(len(keys), P)
    for r in range(P):
        ids = O.mlp_bucket_f32(w, O.mlp_inputs(keys[bounds[r]:bounds[r + 1]], kmin, scale), P)
        for b in range(P + 1):
            assert cut[r, b] == np.count_nonzero(ids < b)


MLP_MUTATIONS = {
    "relu_mask_dropped": ("dz2 = (dy[:, None] * eff[\"w3\"]) * (z2 > 0)", "dz2 = (dy[:, None] * eff[\"w3\"])"),
    "chain_rule_exp_missing": ("g[\"v1\"] = (dz1 * x[:, None]).sum(axis=0) * eff[\"w1\"]",
                               "g[\"v1\"] = (dz1 * x[:, None]).sum(axis=0)"),
    "block_b_sign_lost": ("return np.where(np.arange(MLP_H) < MLP_HALF, 1.0, -1.0)",
                          "return np.where(np.arange(MLP_H) < MLP_HALF, 1.0, 1.0)"),
    "bucket_uses_ceil": ("b = np.floor(f(P) * c).astype(np.int64)", "b = np.ceil(f(P) * c).astype(np.int64)"),
    "adam_bias_uncorrected": ("upd = lr * (mom[k] / (1 - 0.9 ** step)) / (np.sqrt(vel[k] / (1 - 0.999 ** step)) + 1e-8)",
                              "upd = lr * mom[k] / (np.sqrt(vel[k]) + 1e-8)"),
}


@pytest.mark.parametrize("mutation", sorted(MLP_MUTATIONS))
def test_mlp_pins_catch_planted_mistake(mutation):
    src = open(SRC).read()
    old, new = MLP_MUTATIONS[mutation]
    assert src.count(old) == 1
    mod = types.ModuleType("oracle_copy")
    exec(compile(src.replace(old, new), SRC, "exec"), mod.__dict__)
    import tests.test_oracle_mlp as T
    saved = T.O
    T.O = mod
    try:
        failures = 0
        for fn in [T.test_gradient_matches_finite_differences, T.test_first_adam_step_is_lr_times_sign,
                   T.test_identity_network_buckets_are_integer_floor,
                   T.test_effective_weights_are_monotone_and_forward_rises]:
            try:
                fn()
            except Exception:
                failures += 1
        assert failures > 0
    finally:
        T.O = saved
