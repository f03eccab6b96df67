"""Pins for the HyperNEAT substrate oracle: special cases that reduce to
numpy's matrix product, the layered closed form, and invariances."""
import numpy as np

import oracle
from paper_2404_01817_gb300 import workloads as W


def test_one_block_identity_is_a_matrix_product():
    w = W.substrate_weights(1, 3, res=5, layers=2)
    x = W.normal_inputs(2, (3, 4, 25))
    y = oracle.substrate_forward(w, x, hidden_act=1, output_act=0)
    want = np.einsum("gbs,gst->gbt", x.astype(np.float64), w[:, 0].astype(np.float64))
    np.testing.assert_allclose(y, want, rtol=0, atol=1e-12)


def test_three_layers_tanh_and_sigmoid():
    w = W.substrate_weights(3, 2, res=6, layers=3, scale=0.6)
    x = W.normal_inputs(4, (2, 3, 36))
    y = oracle.substrate_forward(w, x, hidden_act=1, output_act=2)
    w64, x64 = w.astype(np.float64), x.astype(np.float64)
    h = np.tanh(np.einsum("gbs,gst->gbt", x64, w64[:, 0]))
    want = 1.0 / (1.0 + np.exp(-np.einsum("gbs,gst->gbt", h, w64[:, 1])))
    np.testing.assert_allclose(y, want, rtol=0, atol=1e-12)


def test_hidden_permutation_and_zero_weights():
    w = W.substrate_weights(5, 2, res=4, layers=3, scale=0.8)
    x = W.normal_inputs(6, (2, 2, 16))
    y = oracle.substrate_forward(w, x)
    perm = np.random.default_rng(7).permutation(16)
    wp = w.copy()
    wp[:, 0] = w[:, 0][:, :, perm]                      # hidden node t' = perm[t]
    wp[:, 1] = w[:, 1][:, perm, :]
    np.testing.assert_allclose(oracle.substrate_forward(wp, x), y, rtol=0, atol=1e-12)
    zero = np.zeros_like(w)
    assert (oracle.substrate_forward(zero, x) == 0).all()                     # tanh(0)
    assert (oracle.substrate_forward(zero, x, output_act=2) == 0.5).all()     # sigmoid(0)
