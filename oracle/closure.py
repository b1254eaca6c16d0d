"""Learned subgrid closure: features, fine-to-coarse restriction and the MLP.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the
product path imports this module.

The paper has no closure; this is the extension its model has a use for: a
pointwise network that adds a correction to the coarse right-hand side,
trained on the difference between a refined run's tendency and the coarse
tendency of the same (restricted) state.  Every piece is a plain definition
written out in float64:

* ``features``  -- per node: the five state variables q_v, their assembled
  gradients d q_v / d x_d (M^-1 DSS(w J d q_v / d x_d), the operator of
  Eqs. 8-12 applied to q_v itself instead of a flux, i.e. the divergence of
  the vector field q_v e_d) and the heating S_theta: 21 values, in the order
  q_0..q_4, dq_0/dx, dq_0/dy, dq_0/dz, dq_1/dx, ..., dq_4/dz, S_theta.
* ``restriction_1d`` / ``restrict`` -- the fine CG field is, inside each fine
  element, the tensor-product Lagrange interpolant on its LGL nodes (Eq. 4);
  its value at a coarse node is that interpolant evaluated there.  Per
  direction this is a matrix (coarse nodes x fine nodes); the 3-D
  restriction applies the three matrices (the interpolant is a tensor
  product).
* the MLP 21 -> 64 -> 64 -> 5 with SiLU, z / (1 + e^-z), after the two
  hidden layers: ``forward``; the mean-squared error and its gradient by the
  chain rule written out layer by layer: ``loss_and_grad``; Adam (Kingma &
  Ba, ICLR 2015) as published: ``adam_step``.
* ``forward_bf16`` -- the inference precision: weights, normalised inputs
  and hidden activations rounded to bfloat16 (round to nearest even from
  float32), biases and sums in wider precision.

Parameter layout (one flat array): W1 [64, 21] row-major (output, input),
b1 [64], W2 [64, 64], b2 [64], W3 [5, 64], b3 [5]; 5893 values.
"""

import numpy as np

from . import euler as E
from . import lgl

SIZES = (21, 64, 64, 5)


def param_count(sizes=SIZES):
    return sum(o * i + o for i, o in zip(sizes[:-1], sizes[1:]))


def unpack(p, sizes=SIZES):
    """[(W, b), ...] views of the flat parameter array."""
    out, k = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        W = p[k:k + o * i].reshape(o, i)
        k += o * i
        b = p[k:k + o]
        k += o
        out.append((W, b))
    return out


# ---------------------------------------------------------------- features

def features(mesh, q, S_theta):
    """[21, Np]: q (5), assembled gradients (15), S_theta (1)."""
    X = np.zeros((21, mesh.Np))
    X[:5] = q
    zero = np.zeros(mesh.Np)
    for v in range(5):
        for d in range(3):
            F = [q[v] if k == d else zero for k in range(3)]
            X[5 + 3 * v + d] = E.divergence(mesh, F)
    X[20] = 0.0 if S_theta is None else S_theta
    return X


# ---------------------------------------------------------------- restriction

def axis_positions(nel, N, lo, hi, periodic):
    """Global node positions along one axis (the mesh's own formula)."""
    xi = lgl.lgl_points(N)
    h = (hi - lo) / nel
    n = N * nel + (0 if periodic else 1)
    g = np.arange(n)
    e = np.minimum(g // N, nel - 1)
    a = g - N * e
    return lo + (e + (xi[a] + 1.0) / 2.0) * h


def restriction_1d(fine, coarse):
    """Matrix [n_coarse, n_fine] evaluating the fine axis interpolant at the
    coarse nodes.  ``fine`` and ``coarse`` are (nel, N, lo, hi, periodic) of
    the same interval."""
    nel_f, N, lo, hi, per = fine
    xi = lgl.lgl_points(N)
    h = (hi - lo) / nel_f
    n_f = N * nel_f + (0 if per else 1)
    xc = axis_positions(*coarse)
    R = np.zeros((xc.size, n_f))
    for c, x in enumerate(xc):
        s = (x - lo) / h
        e = int(np.clip(np.floor(s), 0, nel_f - 1))
        loc = 2.0 * (s - e) - 1.0
        L = lgl.lagrange_eval(xi, loc)[0]
        for a in range(N + 1):
            R[c, (N * e + a) % n_f] += L[a]
    return R


def restrict(fine_axes, coarse_axes, f):
    """Restrict fields f [nv, Np_fine] (x fastest) to the coarse nodes."""
    R = [restriction_1d(fa, ca) for fa, ca in zip(fine_axes, coarse_axes)]
    nf = [r.shape[1] for r in R]
    g = np.asarray(f).reshape(-1, nf[2], nf[1], nf[0])
    g = np.einsum("vzyx,cx->vzyc", g, R[0])
    g = np.einsum("vzyc,by->vzbc", g, R[1])
    g = np.einsum("vzbc,az->vabc", g, R[2])
    return g.reshape(g.shape[0], -1)


# ---------------------------------------------------------------- MLP

def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_prime(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, X, sizes=SIZES):
    """Y [n, out] for inputs X [n, in]; SiLU after every layer but the last."""
    layers = unpack(p, sizes)
    h = np.asarray(X, dtype=np.float64)
    for k, (W, b) in enumerate(layers):
        z = h @ W.T + b
        h = silu(z) if k < len(layers) - 1 else z
    return h


def loss_and_grad(p, X, T, sizes=SIZES):
    """Mean-squared error over all samples and outputs, and its gradient
    with respect to the flat parameters (back-propagation: the chain rule
    applied layer by layer from the output)."""
    layers = unpack(p, sizes)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    hs, zs = [X], []
    h = X
    for k, (W, b) in enumerate(layers):
        z = h @ W.T + b
        zs.append(z)
        h = silu(z) if k < len(layers) - 1 else z
        hs.append(h)
    r = h - T
    loss = float(np.mean(r * r))
    grads = []
    delta = 2.0 * r / r.size                     # dL/dz of the output layer
    for k in range(len(layers) - 1, -1, -1):
        W, _ = layers[k]
        grads.append((delta.T @ hs[k], delta.sum(axis=0)))
        if k > 0:
            delta = (delta @ W) * silu_prime(zs[k - 1])
    g = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads[::-1]])
    return loss, g


def adam_step(p, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step t >= 1); returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) from float32, returned as
    float64 values."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


CLAMP_IN = 8.0


def normalise(X, mean, scale):
    """(x - mean) * scale per feature in float32 (the kernels' order),
    clamped to [-8, 8] (a state outside the training distribution cannot
    drive the network without bound)."""
    X32 = np.asarray(X, dtype=np.float32)
    Xn = (X32 - np.asarray(mean, np.float32)) * np.asarray(scale, np.float32)
    return np.clip(Xn, -CLAMP_IN, CLAMP_IN).astype(np.float64)


def forward_bf16(p, Xn, sizes=SIZES):
    """Inference precision: bfloat16 weights, inputs and hidden activations,
    float64 biases and sums (the kernels accumulate in float32 and evaluate
    SiLU through a hardware tanh approximation, both below the bfloat16
    rounding that follows)."""
    layers = unpack(np.asarray(p, dtype=np.float64), sizes)
    h = bf16(Xn)
    for k, (W, b) in enumerate(layers):
        z = h @ bf16(W).T + np.asarray(b, np.float32).astype(np.float64)
        h = bf16(silu(z)) if k < len(layers) - 1 else z
    return h
