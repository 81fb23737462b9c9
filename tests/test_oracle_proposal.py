"""Pins for the CPU reference of the learned head proposal network: the spectral layer
against closed forms of the truncated Fourier projection, the loss terms against exact
values, the activation against the erf form, the input pooling against constants."""
import math

import numpy as np

from oracle import proposal as oprop

S = oprop.S


def _wave(k1, k2, phase=0.3):
    x, y = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
    return np.cos(2 * np.pi * (k1 * x + k2 * y) / S + phase).reshape(1, S * S, 1)


def _identity_R():
    return np.ones((oprop.M, 1, 1), dtype=complex)


def test_spectral_layer_keeps_retained_modes():
    # with R = 1 on every mode the layer is the projection onto the kept modes: a real
    # wave whose (k1, k2) or (-k1, -k2) is kept comes back unchanged
    for k1, k2 in [(0, 0), (3, 0), (0, 5), (7, 11), (-4, 9), (11, 1), (-11, 11)]:
        v = _wave(k1, k2)
        np.testing.assert_allclose(oprop.spectral_conv(v, _identity_R()), v, atol=1e-12)


def test_spectral_layer_drops_truncated_modes():
    for k1, k2 in [(13, 0), (0, 12), (5, 13), (16, 3), (3, 16), (12, 4)]:
        v = _wave(k1, k2)
        assert np.abs(oprop.spectral_conv(v, _identity_R())).max() < 1e-12


def test_spectral_layer_edge_mode_kept_once():
    # k1 runs over [-12, 11]: of the pair (+-12, 0) only (-12, 0) is kept, and with the
    # k2 = 0 weight of 1 the wave comes back at half amplitude
    v = _wave(12, 0)
    np.testing.assert_allclose(oprop.spectral_conv(v, _identity_R()), 0.5 * v, atol=1e-12)


def test_spectral_layer_phase_shift_by_imaginary_weight():
    # R = i on every mode shifts each retained wave by +90 degrees: cos -> -sin
    v = _wave(2, 3, phase=0.0)
    x, y = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
    want = -np.sin(2 * np.pi * (2 * x + 3 * y) / S).reshape(1, S * S, 1)
    got = oprop.spectral_conv(v, 1j * _identity_R())
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_block_terms_exact_values():
    rng = np.random.default_rng(0)
    K, d = 64, oprop.DELTA
    Q = np.linalg.qr(rng.standard_normal((1024, K)))[0]
    sub, orth = oprop.block_terms(Q, Q)
    assert math.isclose(sub, K * d / (1 + d), rel_tol=1e-9) and orth < 1e-20
    # twice the target: G = 4 I, C^T C = 4 I
    sub, orth = oprop.block_terms(2 * Q, Q)
    assert math.isclose(sub, K * d / (4 + d), rel_tol=1e-9) and math.isclose(orth, 9 * K, rel_tol=1e-12)
    # a block orthogonal to Q: every principal angle is 90 degrees
    Pc = np.linalg.qr(np.hstack([Q, rng.standard_normal((1024, K))]))[0][:, K:]
    sub, orth = oprop.block_terms(Pc, Q)
    assert math.isclose(sub, K, rel_tol=1e-12) and orth < 1e-20


def test_block_terms_principal_angles():
    # Y = Q cos(theta) + Pc sin(theta) column by column: orthonormal, principal angles
    # theta_j, so sub = K - sum cos^2(theta_j) / (1 + delta)
    rng = np.random.default_rng(1)
    K, d = 64, oprop.DELTA
    Q = np.linalg.qr(rng.standard_normal((1024, K)))[0]
    Pc = np.linalg.qr(np.hstack([Q, rng.standard_normal((1024, K))]))[0][:, K:]
    theta = rng.uniform(0, np.pi / 2, K)
    Y = Q * np.cos(theta) + Pc * np.sin(theta)
    sub, orth = oprop.block_terms(Y, Q)
    assert math.isclose(sub, K - np.sum(np.cos(theta) ** 2) / (1 + d), rel_tol=1e-10)
    assert orth < 1e-20


def test_block_terms_invariant_to_column_mixing():
    # sub depends only on span(Y) up to the ridge: a well-conditioned mixing Y S with
    # singular values in [1, 2] moves it by less than K delta
    rng = np.random.default_rng(2)
    K = 64
    Q = np.linalg.qr(rng.standard_normal((1024, K)))[0]
    Y = np.linalg.qr(Q + 0.3 * rng.standard_normal((1024, K)))[0]
    U, _, Vt = np.linalg.svd(rng.standard_normal((K, K)))
    S = U @ np.diag(np.linspace(1, 2, K)) @ Vt
    a, _ = oprop.block_terms(Y, Q)
    b, _ = oprop.block_terms(Y @ S, Q)
    assert abs(a - b) < K * oprop.DELTA


def test_gelu_tanh_form_close_to_erf_form():
    x = np.linspace(-6, 6, 2001)
    exact = 0.5 * x * (1 + np.array([math.erf(t / math.sqrt(2)) for t in x]))
    assert np.abs(oprop.gelu(x) - exact).max() < 1e-3
    assert oprop.gelu(np.array([0.0]))[0] == 0.0


def test_forward_constant_field_gives_node_independent_pooled_input():
    # a constant coefficient field pools to log c at every coarse node; with all
    # weights zero but the bounds bias, the bounds head returns exactly the bias
    p = np.zeros(oprop.COUNT)
    a, n = oprop.OFFSETS["bb"]
    p[a:a + n] = [1.5, -2.0]
    fields = np.full((2, 64, 64), 3.0)
    s, Y = oprop.forward(p, fields)
    np.testing.assert_array_equal(s, [[1.5, -2.0], [1.5, -2.0]])
    assert np.all(Y == 0)
    # lift weight on the pooled channel only: v = log c everywhere
    a, _ = oprop.OFFSETS["Wl"]
    p[a + 0] = 1.0          # Wl[0][0]
    ab, _ = oprop.OFFSETS["Wb"]
    p[ab + 0] = 1.0         # Wb[0][0]: s0 = mean(v[:, 0]) + 1.5 after 4 layers with zero weights
    s, _ = oprop.forward(p, fields)
    # layers with zero spectral and pointwise weights map v to gelu(0) = 0 (layers 1-3)
    # and the last layer to 0, so s0 = bb0
    assert s[0, 0] == 1.5
