"""Plain FP64 reference of the learned Krylov-control network (test
infrastructure only): a 16 -> 64 -> 64 -> 2 perceptron with GELU hidden
activations, x Phi(x) with Phi the standard normal distribution function
(scipy.special.erf as a library primitive), mean squared error on standardised
targets, and its gradient by the chain rule written out layer by layer.
Parameter layout: W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].

The network is an extension of the method: its only counterpart in the paper is
the phi-function solver's choice of the initial substep and Krylov size (Sec. 4,
reference [10]), so the functions below follow no passage of the paper; they
are the textbook definitions written out."""
import numpy as np
from scipy.special import erf

NI, NH, NO = 16, 64, 2
SIZES = [("W1", (NH, NI)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NO, NH)), ("b3", (NO,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    """Split the flat parameter vector by the layout above (the learned choice of
    the initial KIOPS substep, Sec. 4; the network has no paper counterpart)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SIZES:
        size = int(np.prod(shape))
        out[name] = theta[k:k + size].reshape(shape)
        k += size
    return out


def gelu(x):
    """x Phi(x), Phi the standard normal distribution function."""
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    """d/dx of x Phi(x) = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def standardise(X, norm):
    """(X - mean) / std with the stored input normalisation."""
    norm = np.asarray(norm, dtype=np.float64)
    return (np.asarray(X, dtype=np.float64) - norm[:NI]) / norm[NI:2 * NI]


def forward(theta, Xs):
    """Standardised inputs [n, 16] -> standardised outputs [n, 2] and activations."""
    p = unpack(theta)
    z1 = Xs @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (Xs, z1, h1, z2, h2)


def predict(theta, norm, X):
    """Raw features -> raw outputs."""
    norm = np.asarray(norm, dtype=np.float64)
    y, _ = forward(theta, standardise(X, norm))
    return y * norm[2 * NI + NO:] + norm[2 * NI:2 * NI + NO]


def loss_and_grad(theta, norm, X, T):
    """Mean over samples and outputs of the squared error on standardised
    targets, and its gradient with respect to theta."""
    norm = np.asarray(norm, dtype=np.float64)
    Ts = (np.asarray(T, dtype=np.float64) - norm[2 * NI:2 * NI + NO]) / norm[2 * NI + NO:]
    y, (Xs, z1, h1, z2, h2) = forward(theta, standardise(X, norm))
    p = unpack(theta)
    n = Xs.shape[0]
    r = y - Ts
    loss = np.sum(r * r) / (n * NO)
    dy = 2.0 * r / (n * NO)
    g = {"W3": dy.T @ h2, "b3": dy.sum(axis=0)}
    dz2 = (dy @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ Xs
    g["b1"] = dz1.sum(axis=0)
    return loss, np.concatenate([g[name].reshape(-1) for name, _ in SIZES])
