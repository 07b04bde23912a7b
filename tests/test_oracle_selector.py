"""Pins for the selector's CPU oracles (oracle/mlp.py, oracle/features.py):
finite differences for the gradient, hand-computed outputs of sparse
parameter sets, Adam's closed-form first step, and features of matrices
whose features are known by construction."""
import numpy as np

import gen
from oracle import features as F
from oracle import mlp


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, mlp.H * mlp.IN + mlp.H + mlp.H * mlp.H + mlp.H + mlp.OUT * mlp.H + mlp.OUT)
    x = rng.normal(0, 1, (7, mlp.IN))
    t = rng.normal(0, 1, (7, mlp.OUT))
    mask = (rng.random((7, mlp.OUT)) < 0.7).astype(float)
    out, cache = mlp.forward(p, x)
    L0, dout = mlp.loss(out, t, mask)
    g = mlp.backward(p, cache, dout)
    for k in rng.choice(p.size, 60, replace=False):
        e = np.zeros_like(p)
        e[k] = 1e-6
        lp, _ = mlp.loss(mlp.forward(p + e, x)[0], t, mask)
        lm, _ = mlp.loss(mlp.forward(p - e, x)[0], t, mask)
        assert abs((lp - lm) / 2e-6 - g[k]) <= 1e-6 * max(1.0, abs(g[k]))


def test_mlp_forward_hand_computed():
    # one path: x[5] -(W1[3][5]=2)-> h1[3] -(W2[7][3]=-0.5, b2[7]=4)-> h2[7] -(W3[2][7]=3)-> out[2]
    W1, b1, W2, b2, W3, b3 = (np.zeros((64, 22)), np.zeros(64), np.zeros((64, 64)),
                              np.zeros(64), np.zeros((mlp.OUT, 64)), np.zeros(mlp.OUT))
    W1[3, 5] = 2.0
    W2[7, 3] = -0.5
    b2[7] = 4.0
    W3[2, 7] = 3.0
    b3[:] = np.arange(mlp.OUT)
    p = mlp.pack([W1, b1, W2, b2, W3, b3])
    x = np.zeros((3, 22))
    x[0, 5] = 1.0    # h1 = 2, h2 = relu(-1 + 4) = 3, out[2] = 9 + 2
    x[1, 5] = -1.0   # h1 = relu(-2) = 0, h2 = 4, out[2] = 12 + 2
    x[2, 5] = 10.0   # h1 = 20, h2 = relu(-10 + 4) = 0, out[2] = 0 + 2
    out, _ = mlp.forward(p, x)
    assert np.allclose(out[:, 2], [11.0, 14.0, 2.0])
    others = [k for k in range(mlp.OUT) if k != 2]
    assert np.allclose(out[:, others], np.arange(mlp.OUT)[others])


def test_adam_first_step_is_lr_sign():
    rng = np.random.default_rng(1)
    p = rng.normal(size=100)
    g = rng.normal(size=100)
    p1, m, v = mlp.adam_step(p, g, np.zeros(100), np.zeros(100), 1, lr=0.01, eps=0.0)
    assert np.allclose(p1, p - 0.01 * np.sign(g))


def test_bin_of_length():
    L = np.array([0, 1, 2, 3, 4, 5, 8, 9, 16, 17, 32768, 32769, 10 ** 6])
    assert list(F.bin_of_length(L)) == [0, 1, 2, 3, 3, 4, 4, 5, 5, 6, 16, 16, 16]


def test_features_of_identity_and_empty():
    n = 1000
    I = gen.dense_to_csr(np.eye(n, dtype=np.int64), 65521)
    f, g = F.features(I.nrows, I.ncols, I.row_ptr, I.col, I.val, I.modulus)
    assert f[2] == np.log2(2) / 16 and f[3] == 0 and f[5] == 0 and f[6] == 1 and f[7] == 0
    assert f[8] == 1          # every value is 1
    assert f[10] == 1 and f[11] == 1 and f[12] == 1 and f[13] == 0 and f[15] == 1
    assert g[1][1] == 1 and g[1][2] == 1 and g[1][3] == 1 and g[1][4] == 1
    E = gen.CSR(10, 7, np.zeros(11, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint32), 3)
    f, g = F.features(E.nrows, E.ncols, E.row_ptr, E.col, E.val, E.modulus)
    assert f[5] == 1 and f[8] == 0 and f[15] == 0 and g[0][1] == 1


def test_features_of_a_row_split():
    # rows of lengths 1, 3, 64 and one empty row; +-1 only in the long row
    m = 7
    lengths = np.array([1, 3, 64, 0])
    cols = np.concatenate([np.arange(L) for L in lengths]).astype(np.int32)
    vals = np.concatenate([[2], [3, 4, 5], np.full(64, 6)]).astype(np.uint32)   # 6 = -1 mod 7
    A = gen.CSR(4, 100, np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64), cols, vals, m)
    f, g = F.features(A.nrows, A.ncols, A.row_ptr, A.col, A.val, m)
    mean = 68 / 4
    assert np.isclose(f[2], np.log2(1 + mean) / 16)
    assert f[5] == 0.25 and f[6] == 0.5 and f[7] == 0.25 and np.isclose(f[8], 64 / 68)
    assert np.isclose(g[7][3], 1.0) and g[2][3] == 0 and np.isclose(g[7][4], 1.0)   # 64 -> bin 7
    assert np.isclose(g[3][4], 3 / 4)
