"""Learned covariance surrogate (oracle; test infrastructure only).

The paper has no learned component.  Its applications of camera covariances
(Sec. 1: next-best-view selection, detecting badly added cameras, filtering
unconstrained cameras) motivate a cheap per-camera predictor; this module
states that predictor in plain numpy so that the CUDA kernels can be checked
against it.

Model, per camera i of a scene:
  Z_ii    the 9x9 diagonal block of the reduced camera matrix of Sec. 4.2,
          Z = U - W A^-1 W^T, i.e. U_i - sum over the camera's observations
          of W_ij A_j^-1 W_ij^T;
  d       sqrt(diag Z_ii) (9 values), the block's Jacobi scale;
  L_z     the Cholesky factor of Z_ii (Z_ii = L_z L_z^T): Z_ii^-1 is the
          covariance the camera would have with every other camera fixed;
  features (64 values):
          [0, 36)   C_kl = Z_kl / (d_k d_l) for k < l, row by row
          [36, 45)  log d_k
          45        log of the camera's observation count
          46        mean over its observations of log L_j (L_j = track length)
          47        fraction of its observations with L_j = 2
          48        10 / sqrt(n), n the cameras in the scene (around the base
                    with the gauge term below, what remains shrinks about as
                    n^-1/2, so a network that is linear in this feature
                    beyond the training sizes follows it to larger scenes)
          49        |c_i - c_mean| / rms radius of the camera centres c = -R^T t
          [50, 64)  zero
  target  (45 values): the Cholesky factor L of the whitened exact block
          S = L_z^T Sigma_i L_z (S = I when Sigma_i = Z_ii^-1):
          [0, 9) log L_kk, [9, 45) L_kl for k > l, row by row;
  output  Sigma_hat_i = L_z^-T L_hat L_hat^T L_z^-1, L_hat from a network
          output in the target's form, so that the network learns how far the
          whole scene moves the camera's covariance away from Z_ii^-1.

Gauge term of the base.  Z_ii^-1 holds every other camera fixed, which also
pins the datum; in the similarity gauge of Sec. 4.1 the camera moves with
the datum as well.  On the exact blocks of the shell scenes the difference
Sigma_i - Z_ii^-1 lies almost entirely (over 99% of its whitened squared
norm) in the span of the camera's nullspace rows H_i (the 9 x 7 rows of H
for camera i, Sec. 4.1), and one 7 x 7 matrix per scene explains nearly all
of that part.  In the scene's own metric that matrix hardly
depends on the scene's size, so one learned M serves all sizes:
  AH      sum_i H_i^T Z_ii H_i (7 x 7), L_c the Cholesky factor of AH^-1
  Q_i     H_i L_c (9 x 7), so that sum_i Q_i^T Z_ii Q_i = I
  B_i     Z_ii^-1 + Q_i M Q_i^T, the base covariance (M = 0: Z_ii^-1)
  T_i     the Cholesky factor of B_i^-1 (M = 0: L_z)
  M       symmetric 7 x 7, least squares over the training cameras of
          |L_z^T (Sigma_i - Z_ii^-1) L_z - L_z^T Q_i M Q_i^T L_z|_F^2.
Targets and outputs are then taken with T_i in place of L_z: the network
learns the remainder of the scene's effect beyond the gauge term.

Network: 64 -> 256 -> 256 -> 256 -> 45, ReLU after the three hidden layers,
inputs and targets standardised with per-column mean and standard deviation
of the training set (a deviation below 1e-6 is replaced by 1).  The output
head carries a size scale s = feature 48 (10 / sqrt(n); 1 if that feature
is not positive): the network learns the standardised t / s, and its output
y stands for t = s (mu_t + sd_t y), the target normalisation being taken on
t / s.  Around the base with the gauge term the remainder shrinks about as
n^-1/2 (60-1000 cameras), so t / s keeps its size from scene to scene and
the network need not extrapolate in the scene's size.  Feature 48 sets only
that scale: its standardised input column is zero (every other feature has
the same distribution at 60 and at 2000 cameras, so no input leaves the
training range on larger scenes).  Loss: mean
squared error over the 45 standardised outputs and the batch.  Optimiser:
Adam (Kingma and Ba, 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8.

Precision: the kernels multiply bf16 operands with fp32 accumulation.  The
functions below take `quantize`; when it is set, every GEMM operand is
rounded to bf16 (round to nearest even) at the same points as the kernels:
the standardised inputs, the weights, the hidden activations after ReLU, and
the output-side gradients fed to the two backward products.  Biases, the
output, the loss and every sum stay in float64 here (fp32 on the GPU).  With
`quantize` off the functions are the exact float64 gradient of the loss.

Parity: gauge rows pinned by their normalisation (sum_i Q_i^T Z_ii Q_i = I)
and by their span; the base factor by M = 0 (T = L_z) and by the push-through
form of B^-1; the gauge fit by recovery of a planted M and by the optimality
condition of least squares; forward/backward pinned by finite differences and by torch autograd
in float64; Adam by torch.optim.Adam; bf16 rounding by torch's conversion;
features by the dense Schur complement of `covariance` and by brute-force
counting; targets by the round trip back to Sigma and by the closed form
Sigma = Z_ii^-1 -> S = I; the KL measure by its closed form for scaled
identities.
"""
from __future__ import annotations

import numpy as np

from . import camera, information

F_IN, HIDDEN, F_OUT = 64, 256, 45
DIMS = (F_IN, HIDDEN, HIDDEN, HIDDEN, F_OUT)
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8
_IU = np.triu_indices(9, 1)       # (k, l), k < l, row by row
_IL = np.tril_indices(9, -1)      # (k, l), k > l, row by row


def param_shapes():
    """[(out, in), (out,)] per layer, in the packing order W1, b1, ..., W4, b4."""
    out = []
    for a, b in zip(DIMS[:-1], DIMS[1:]):
        out += [(b, a), (b,)]
    return out


def n_params() -> int:
    return sum(int(np.prod(s)) for s in param_shapes())


def unpack(flat: np.ndarray) -> list:
    out, o = [], 0
    for s in param_shapes():
        k = int(np.prod(s))
        out.append(np.asarray(flat[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def pack(arrs) -> np.ndarray:
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in arrs])


# ---------------------------------------------------------------------------
# bf16 rounding: keep the 8 leading significand bits of the float32 value,
# round to nearest, ties to even.
def bf16(x: np.ndarray) -> np.ndarray:
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


# ---------------------------------------------------------------------------
# Features and targets
def diagonal_blocks(scene) -> np.ndarray:
    """Z_ii = U_i - sum_{j seen by i} W_ij A_j^-1 W_ij^T, (n, 9, 9)."""
    U, A, W, _, _ = information.blocks(scene)
    Ainv = np.linalg.inv(A)
    Z = U.copy()
    for o in range(scene.t):
        i, j = scene.obs_cam[o], scene.obs_pt[o]
        Z[i] -= W[o] @ Ainv[j] @ W[o].T
    return Z


def degree_stats(scene) -> np.ndarray:
    """(n, 3): log #obs, mean log track length, fraction of 2-tracks."""
    L = np.bincount(scene.obs_pt, minlength=scene.m)
    out = np.zeros((scene.n, 3))
    for i in range(scene.n):
        tr = L[scene.obs_pt[scene.obs_cam == i]]
        out[i] = [np.log(len(tr)), np.mean(np.log(tr)), np.mean(tr == 2)]
    return out


def centre_distance(scene) -> np.ndarray:
    c = np.stack([-camera.rotation_matrix(p[:3]).T @ p[3:6] for p in scene.cams])
    dev = c - c.mean(axis=0)
    rms = np.sqrt(np.mean(np.sum(dev ** 2, axis=1)))
    return np.sqrt(np.sum(dev ** 2, axis=1)) / rms


def features(scene):
    """(features (n, 64), L_z (n, 9, 9) lower triangular)."""
    Z = diagonal_blocks(scene)
    d = np.sqrt(np.einsum("ikk->ik", Z))
    C = Z / (d[:, :, None] * d[:, None, :])
    f = np.zeros((scene.n, F_IN))
    f[:, :36] = C[:, _IU[0], _IU[1]]
    f[:, 36:45] = np.log(d)
    f[:, 45:48] = degree_stats(scene)
    f[:, 48] = 10.0 / np.sqrt(scene.n)
    f[:, 49] = centre_distance(scene)
    return f, np.linalg.cholesky(Z)


def targets(sigma: np.ndarray, Lz: np.ndarray) -> np.ndarray:
    """Cholesky form of S = L_z^T Sigma L_z, (n, 45)."""
    S = Lz.transpose(0, 2, 1) @ sigma @ Lz
    L = np.linalg.cholesky(S)
    return np.concatenate([np.log(np.einsum("ikk->ik", L)), L[:, _IL[0], _IL[1]]], axis=1)


def covariance_from_output(t: np.ndarray, Lz: np.ndarray) -> np.ndarray:
    """Sigma_hat = L_z^-T L L^T L_z^-1 from outputs in the target form."""
    n = t.shape[0]
    L = np.zeros((n, 9, 9))
    k = np.arange(9)
    L[:, k, k] = np.exp(t[:, :9])
    L[:, _IL[0], _IL[1]] = t[:, 9:]
    Li = np.linalg.inv(Lz)
    return Li.transpose(0, 2, 1) @ (L @ L.transpose(0, 2, 1)) @ Li


# ---------------------------------------------------------------------------
# Gauge term of the base covariance
def gauge_rows(Lz: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Q_i = H_i L_c (n, 9, 7) for one scene: Lz (n, 9, 9) the factors of the
    blocks Z_ii, H (n, 9, 7) the cameras' nullspace rows, L_c the Cholesky
    factor of (sum_i H_i^T Z_ii H_i)^-1."""
    Zd = Lz @ Lz.transpose(0, 2, 1)
    AH = np.einsum("iak,iab,ibl->kl", H, Zd, H)
    Lc = np.linalg.cholesky(np.linalg.inv(AH))
    return H @ Lc


def base_factor(Lz: np.ndarray, Q: np.ndarray, M: np.ndarray) -> np.ndarray:
    """T_i = chol((Z_ii^-1 + Q_i M Q_i^T)^-1), (n, 9, 9) lower triangular."""
    Zinv = np.linalg.inv(Lz @ Lz.transpose(0, 2, 1))
    B = Zinv + Q @ M @ Q.transpose(0, 2, 1)
    return np.linalg.cholesky(np.linalg.inv(B))


def sym_basis() -> np.ndarray:
    """The 28 symmetric 7 x 7 matrices E_kl (k <= l, row by row): ones at
    (k, l) and (l, k).  M = sum over k <= l of M_kl E_kl."""
    out = []
    for k in range(7):
        for l in range(k, 7):
            E = np.zeros((7, 7))
            E[k, l] = E[l, k] = 1.0
            out.append(E)
    return np.stack(out)


def fit_gauge(Lz: np.ndarray, Q: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """The symmetric M that minimises, over the given cameras (of any number
    of scenes, each Q from its own scene),
        sum_i |L_z^T (Sigma_i - Z_ii^-1) L_z - L_z^T Q_i M Q_i^T L_z|_F^2
    (L_z^T Z_ii^-1 L_z = I): linear least squares in the 28 entries M_kl,
    k <= l."""
    Qt = Lz.transpose(0, 2, 1) @ Q
    E = Lz.transpose(0, 2, 1) @ sigma @ Lz - np.eye(9)
    A = np.stack([Qt @ Eb @ Qt.transpose(0, 2, 1) for Eb in sym_basis()], axis=-1)
    m = np.linalg.lstsq(A.reshape(-1, 28), E.reshape(-1), rcond=None)[0]
    return np.einsum("p,pkl->kl", m, sym_basis())


def gaussian_kl(pred: np.ndarray, true: np.ndarray) -> np.ndarray:
    """KL(N(0, true) || N(0, pred)) per block: an error measure of a
    covariance that does not depend on the units of the parameters."""
    Pi = np.linalg.inv(pred)
    return 0.5 * (np.einsum("iab,iba->i", Pi, true) - true.shape[1] + np.linalg.slogdet(pred)[1]
                  - np.linalg.slogdet(true)[1])


def normalization(x: np.ndarray):
    """Column mean and deviation (population), deviation < 1e-6 -> 1."""
    mu = x.mean(axis=0)
    sd = np.sqrt(np.mean((x - mu) ** 2, axis=0))
    return mu, np.where(sd < 1e-6, 1.0, sd)


# ---------------------------------------------------------------------------
# Network
def forward(params, x, quantize=True):
    """x: standardised inputs (B, 64).  Returns (y (B, 45), activations a0..a3)."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    W = params[0::2]
    b = params[1::2]
    acts = [q(x)]
    for layer in range(3):
        z = acts[-1] @ q(W[layer]).T + b[layer]
        acts.append(q(np.maximum(z, 0.0)))
    y = acts[-1] @ q(W[3]).T + b[3]
    return y, acts


def loss_and_grads(params, x, t, quantize=True):
    """Mean squared error over the batch and the 45 outputs, and its gradients
    with respect to [W1, b1, ..., W4, b4] (straight-through at the bf16
    roundings when `quantize` is set)."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    y, acts = forward(params, x, quantize)
    B = x.shape[0]
    r = y - t
    loss = float(np.sum(r * r) / (B * F_OUT))
    g = 2.0 * r / (B * F_OUT)                     # dL/dz of the output layer
    W = params[0::2]
    grads = [None] * 8
    for layer in range(3, -1, -1):
        grads[2 * layer] = q(g).T @ acts[layer]
        grads[2 * layer + 1] = g.sum(axis=0)
        if layer > 0:
            dx = q(g) @ q(W[layer])
            g = dx * (acts[layer] > 0)
    return loss, grads


def adam(params, grads, m, v, step, lr):
    """One Adam step (step counts from 1); returns new params, m, v."""
    out_p, out_m, out_v = [], [], []
    c1 = 1.0 - BETA1 ** step
    c2 = 1.0 - BETA2 ** step
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = BETA1 * mm + (1.0 - BETA1) * g
        vv = BETA2 * vv + (1.0 - BETA2) * g * g
        p = p - lr * (mm / c1) / (np.sqrt(vv / c2) + EPS)
        out_p.append(p)
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v


def network_input(f: np.ndarray, mu_f: np.ndarray, sd_f: np.ndarray) -> np.ndarray:
    """Standardised features with the size feature's column set to zero."""
    x = (f - mu_f) / sd_f
    x[:, 48] = 0.0
    return x


def head_scale(f: np.ndarray) -> np.ndarray:
    """The output head's size scale per row of raw features f (n, 64)."""
    return np.where(f[:, 48] > 0, f[:, 48], 1.0)


def predict(params, f, Lz, norm, quantize=True):
    """Sigma_hat for raw features f (n, 64) with normalisation (mu_f, sd_f, mu_t, sd_t)
    and whitening factors Lz (L_z, or the base factors T)."""
    mu_f, sd_f, mu_t, sd_t = norm
    y, _ = forward(params, network_input(f, mu_f, sd_f), quantize)
    return covariance_from_output(head_scale(f)[:, None] * (y * sd_t + mu_t), Lz)
