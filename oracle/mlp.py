"""FP64 CPU oracle of the warm-start network (test infrastructure only).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.  It shares no code with the CUDA library.

The paper has no learned component; this is the small multilayer perceptron that maps
the parameters of a run, (a, T/T_c, sigma, viscosity ratio), to the equilibrium
quantities used to initialise droplets and films (coexistence densities and the tanh
profile of Eq. 31).  Everything here is the textbook definition, written out plainly:

  layers     4 -> 64 -> 64 -> 5, affine maps y = W x + b, W stored (out, in) row-major.
  gelu       x * Phi(x), Phi the standard normal CDF (Hendrycks & Gimpel 2016), by erfc
             (Phi(x) = erfc(-x / sqrt 2) / 2 has no cancellation for negative x).
  loss       mean over rows and outputs of the squared error of the standardised output.
  gradient   reverse-mode chain rule through the three layers.
  adam       Kingma & Ba (2015), Algorithm 1, with bias-corrected moment estimates.
  bf16       round-to-nearest-even of an FP32 value to 8 mantissa bits (the weight copy
             the forward and backward passes read; accumulation stays in FP64 here).

Parameter vector packing (NPARAMS = 4805): W1 (64, 4), b1 (64), W2 (64, 64), b2 (64),
W3 (5, 64), b3 (5).  Inputs are standardised with (x - in_mean) / in_scale before the
first layer; the network output is in standardised units, out_mean + out_scale * y in
physical ones.
"""
import math

import numpy as np

N_IN, N_HID, N_OUT = 4, 64, 5
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)),
          ("b2", (N_HID,)), ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)

_erfc = np.vectorize(math.erfc, otypes=[np.float64])


def _phi_cdf(z):
    return 0.5 * _erfc(-z / math.sqrt(2.0))


def unpack(p):
    """Views of the packed parameter vector as the six named arrays."""
    p = np.asarray(p, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[k:k + n].reshape(shape)
        k += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(z):
    """z * Phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return z * _phi_cdf(z)


def gelu_grad(z):
    """d gelu / dz = Phi(z) + z phi(z), phi the standard normal density."""
    z = np.asarray(z, dtype=np.float64)
    return _phi_cdf(z) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.  The value is
    first rounded to float32, as the master weights are held in FP32."""
    b = np.asarray(x, dtype=np.float32).astype(np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def fit_scaling(x, t):
    """Per-column mean and standard deviation (population form, ones where a column is
    constant) of the inputs x (n, 4) and targets t (n, 5)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)

    def ms(a):
        mu = a.mean(axis=0)
        sd = a.std(axis=0)
        return mu, np.where(sd > 0, sd, 1.0)

    im, isd = ms(x)
    om, osd = ms(t)
    return {"in_mean": im, "in_scale": isd, "out_mean": om, "out_scale": osd}


def forward(p, x, scaling, weights=None):
    """Standardised outputs (n, 5) and the intermediate values the backward pass needs.
    weights: None for the parameters as given, "bf16" to evaluate with bf16-rounded
    weights and biases."""
    P = unpack(bf16_round(p) if weights == "bf16" else p)
    xn = (np.asarray(x, dtype=np.float64) - scaling["in_mean"]) / scaling["in_scale"]
    z1 = xn @ P["W1"].T + P["b1"]
    h1 = gelu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(z2)
    y = h2 @ P["W3"].T + P["b3"]
    return y, {"P": P, "xn": xn, "z1": z1, "h1": h1, "z2": z2, "h2": h2}


def predict(p, x, scaling, weights=None):
    y, _ = forward(p, x, scaling, weights)
    return scaling["out_mean"] + scaling["out_scale"] * y


def loss(p, x, t, scaling, weights=None):
    y, _ = forward(p, x, scaling, weights)
    tn = (np.asarray(t, dtype=np.float64) - scaling["out_mean"]) / scaling["out_scale"]
    return float(np.mean((y - tn) ** 2))


def gradient(p, x, t, scaling, weights=None):
    """(loss, dloss/dp packed like p).  With weights="bf16" the derivative is taken at the
    rounded weights (rounding is treated as the identity, as in training)."""
    y, c = forward(p, x, scaling, weights)
    P = c["P"]
    tn = (np.asarray(t, dtype=np.float64) - scaling["out_mean"]) / scaling["out_scale"]
    n = y.shape[0]
    dy = 2.0 * (y - tn) / (n * N_OUT)
    g = {"W3": dy.T @ c["h2"], "b3": dy.sum(axis=0)}
    dz2 = (dy @ P["W3"]) * gelu_grad(c["z2"])
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"]) * gelu_grad(c["z1"])
    g["W1"] = dz1.T @ c["xn"]
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean((y - tn) ** 2)), pack(g)


def adam_step(p, g, m, v, k, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step number k >= 1; returns
    the new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** k)
    vhat = v / (1.0 - beta2 ** k)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(p0, x, t, scaling, steps, lr, beta1=0.9, beta2=0.999, eps=1e-8, weights="bf16"):
    """Full-batch Adam from p0 for `steps` updates; returns (p, losses) where losses[k] is
    the loss at the weights used by update k + 1."""
    p = np.asarray(p0, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for k in range(1, steps + 1):
        L, g = gradient(p, x, t, scaling, weights)
        losses.append(L)
        p, m, v = adam_step(p, g, m, v, k, lr, beta1, beta2, eps)
    return p, np.array(losses)
