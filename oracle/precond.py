"""FP64 oracle of the learned element-wise preconditioner (test infrastructure only).

Not a paper operator: the spec preconditioner for CG over the
matrix-free operator, restated here in plain numpy:

    M(r) = D^{-1} r + sum_K R_K^T ( w_K * s_K * f(R_K r / s_K) ),
    f(z) = W2 relu(W1 z + b1),   s_K = ||R_K r||_2   (contribution 0 if s_K = 0),

R_K gathers the cell's local dofs, w_K holds 1 / (number of cells sharing
each node) at the cell's nodes, D is the operator diagonal.  Training
minimises L = (M(r) - e)^T A (M(r) - e) / (e^T A e) over (residual, error)
pairs; `loss_and_grad` returns L and its exact gradient by backpropagation
through the MLP, the scaling, and the assembly.

Operand precision.  The network's weights are BF16 (the caller passes them
rounded), and the kernels that evaluate it multiply BF16 operands with FP32
accumulation: the normalised inputs Z and the hidden activations H in the
forward pass, dL/dO and dL/dH in the backward pass.  `rnd`, when given, is
applied to exactly those four operands, so that a test can compare a kernel
with this oracle at the kernel's operand precision; the default (None) keeps
everything in FP64.  It rounds values only: the order of the steps is the same.
"""
import numpy as np


def multiplicity_weights(cell_node, nnode):
    mult = np.bincount(cell_node.ravel(), minlength=nnode).astype(np.float64)
    return 1.0 / np.maximum(mult, 1.0)


def _keep(a):
    return a


def apply(r, cell_node, winv, dinv, W1, b1, W2, rnd=None):
    """M(r) in FP64.  W1 [H][nloc], b1 [H], W2 [nloc][H]; rnd: operand rounding (module docstring)."""
    rnd = rnd or _keep
    out = dinv * r
    R = r[cell_node]                      # [ncell][nloc]
    s = np.linalg.norm(R, axis=1)         # [ncell]
    safe = np.where(s > 0, s, 1.0)
    Z = rnd(R / safe[:, None])
    Hpre = Z @ W1.T + b1
    H = rnd(np.maximum(Hpre, 0.0))
    O = H @ W2.T                          # [ncell][nloc]
    contrib = winv[cell_node] * (s[:, None] * O) * (s[:, None] > 0)
    np.add.at(out, cell_node, contrib)
    return out


def loss_and_grad(r, e, A_apply, cell_node, winv, dinv, W1, b1, W2, rnd=None):
    """Loss L and (dL/dW1, dL/db1, dL/dW2) for one pair; A_apply(v) = A v; rnd as for `apply`."""
    rnd = rnd or _keep
    R = r[cell_node]
    s = np.linalg.norm(R, axis=1)
    safe = np.where(s > 0, s, 1.0)
    Z = rnd(R / safe[:, None])
    Hpre = Z @ W1.T + b1
    H = rnd(np.maximum(Hpre, 0.0))
    O = H @ W2.T
    alive = (s > 0)[:, None]
    M = dinv * r
    np.add.at(M, cell_node, winv[cell_node] * (s[:, None] * O) * alive)
    u = M - e
    Au = A_apply(u)
    den = e @ A_apply(e)
    L = (u @ Au) / den
    g = 2.0 * Au / den                    # dL/du (A symmetric)
    Delta = rnd(winv[cell_node] * g[cell_node] * s[:, None] * alive)  # dL/dO
    dW2 = Delta.T @ H
    dH = rnd((Delta @ W2) * (H > 0))
    dW1 = dH.T @ Z
    db1 = dH.sum(axis=0)
    return L, dW1, db1, dW2


# ---- linear (tied, symmetric) variant:
#   M(r) = D^{-1} r + sum_K R_K^T w_K W1^T W1 (w_K R_K r)

def apply_linear(r, cell_node, winv, dinv, W1, rnd=None):
    """M(r) of the linear variant; rnd: operand rounding of Z and H (module docstring)."""
    rnd = rnd or _keep
    out = dinv * r
    Z = rnd(winv[cell_node] * r[cell_node])
    O = rnd(Z @ W1.T) @ W1
    np.add.at(out, cell_node, winv[cell_node] * O)
    return out


def loss_and_grad_linear(r, e, A_apply, cell_node, winv, dinv, W1):
    """L = (M r - e)^T A (M r - e) / (e^T A e) and dL/dW1 for the linear variant."""
    Z = winv[cell_node] * r[cell_node]
    H = Z @ W1.T
    O = H @ W1
    M = dinv * r
    np.add.at(M, cell_node, winv[cell_node] * O)
    u = M - e
    Au = A_apply(u)
    den = e @ A_apply(e)
    L = (u @ Au) / den
    g = 2.0 * Au / den
    Delta = winv[cell_node] * g[cell_node]      # dL/dO
    dW1 = H.T @ Delta + (Delta @ W1.T).T @ Z     # O = W1^T (W1 z)
    return L, dW1
