"""CPU FP64 reference of the packing MLP -- TEST INFRASTRUCTURE ONLY.

16 -> 64 -> 64 -> 1 with ReLU, loss = mean (f(x) - y)^2, written from the
definition of the forward pass and the chain rule (no library autodiff).
Parameter layout: W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3.
"""
import numpy as np

IN, H = 16, 64
SIZES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
NP = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    w = np.asarray(w, np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = w[o:o + n].reshape(shape)
        o += n
    return out


def forward(w, x):
    p = unpack(w)
    x = np.asarray(x, np.float64)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (x, a1, h1, a2, h2)


def loss_and_grad(w, x, t):
    """mean squared error and its gradient with respect to the flat weights"""
    p = unpack(w)
    y, (x, a1, h1, a2, h2) = forward(w, x)
    t = np.asarray(t, np.float64)
    n = len(t)
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / n
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dh2 = np.outer(dy, p["w3"]) * (a2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ p["W2"]) * (a1 > 0)
    g["W1"] = dh1.T @ x
    g["b1"] = dh1.sum(0)
    return loss, np.concatenate([g[name].ravel() for name, _ in SIZES])


def init(seed):
    rng = np.random.default_rng(seed)
    w = []
    for name, shape in SIZES:
        n = int(np.prod(shape))
        if name.startswith("W") or name == "w3":
            fan = shape[-1] if name != "w3" else H
            w.append(rng.uniform(-1, 1, n) * np.sqrt(6.0 / fan))
        else:
            w.append(np.zeros(n))
    return np.concatenate(w)
