"""CPU reference of the warm-start MLP (test infrastructure only).

A plain numpy restatement of a fully connected network with ReLU between
layers, its mean-squared-error loss and the loss's gradient by the chain rule
(reverse mode written out layer by layer).  Parameters use the library's flat
layout: per layer l, W_l (dims[l] x dims[l+1], row-major) then b_l.  The
computation runs in the dtype of the inputs (float32 for the parity checks,
float64 for the finite-difference pins).  The paper has no learned
component, so nothing in it pins this code; it is pinned by central finite
differences of the loss, by the least-squares optimum of a single linear
layer, where the gradient must vanish, and its bfloat16 rounding by a library
float32 -> bfloat16 conversion.
"""
import numpy as np


def unpack(theta, dims):
    """Split the flat parameter vector into [(W_l, b_l)]."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        a, b = dims[l], dims[l + 1]
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        bias = theta[o:o + b]
        o += b
        out.append((W, bias))
    assert o == len(theta)
    return out


def round_bf16(a):
    """float32 -> nearest bfloat16 (ties to even), returned as float32: the
    8-bit-exponent, 8-bit-significand format keeps the top 16 bits."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def _q(a, bf16):
    return round_bf16(a) if bf16 else a


def forward(theta, dims, x, bf16=False):
    """Returns the output and the pre-activations of every layer.  With
    bf16=True the operands of every product (inputs, weights, hidden
    activations) are rounded to bfloat16 first, as the tensor-core path
    stores them; sums stay in the input dtype."""
    layers = unpack(theta, dims)
    h, zs = _q(x, bf16), []
    for l, (W, b) in enumerate(layers):
        z = h @ _q(W, bf16) + b
        zs.append(z)
        h = _q(np.maximum(z, 0), bf16) if l + 1 < len(layers) else z
    return h, zs


def loss_and_grad(theta, dims, x, t, bf16=False):
    """Mean squared error over all output entries and its gradient.  With
    bf16=True the back-propagated output gradient and every propagated
    hidden gradient are rounded to bfloat16 as well."""
    layers = unpack(theta, dims)
    y, zs = forward(theta, dims, x, bf16)
    n = y.size
    d = y - t
    loss = float(np.sum(d * d) / n)
    dz = _q((2.0 / n) * d, bf16)
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        h_in = _q(x, bf16) if l == 0 else _q(np.maximum(zs[l - 1], 0), bf16)
        grads.append((h_in.T @ dz, dz.sum(axis=0)))
        if l > 0:
            dz = _q((dz @ _q(W, bf16).T) * (zs[l - 1] > 0), bf16)
    grads.reverse()
    return loss, np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads]).astype(theta.dtype)


def grad_abs_scale(theta, dims, x, t, bf16=False):
    """Per gradient entry, the sum of the magnitudes of the products that make
    it up (|h_in|^T |dz| for a weight, sum |dz| for a bias), with |dz| back
    propagated through |W|: the scale of the entry's rounding error, since a
    rounding change of one operand moves the entry by at most that operand's
    relative change times this sum.  Same flat layout as the gradient."""
    layers = unpack(theta, dims)
    y, zs = forward(theta, dims, x, bf16)
    n = y.size
    dz = np.abs(_q((2.0 / n) * (y - t), bf16))
    out = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        h_in = np.abs(_q(x, bf16) if l == 0 else _q(np.maximum(zs[l - 1], 0), bf16))
        out.append((h_in.T @ dz, dz.sum(axis=0)))
        if l > 0:
            dz = (dz @ np.abs(_q(W, bf16)).T) * (zs[l - 1] > 0)
    out.reverse()
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in out]).astype(theta.dtype)
