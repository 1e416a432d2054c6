"""FP64 CPU oracle of the learned surrogate's network (test infrastructure only).

Plain numpy, float64, written from the definition of the network the library trains:
x_n = (x - shift) * scale; h1 = silu(W1 x_n + b1); h2 = silu(W2 h1 + b2);
h3 = silu(W3 h2 + b3); out = W4 h3 + b4; loss = mean over rows and the 6 used outputs of
(out - (y - mu)/sigma)^2.  Parameters use the library's flat layout: W1[256][4], b1,
W2[256][256], b2, W3[256][256], b3, W4[8][256], b4[8], then 24 normalisation constants
(input scale[4], shift[4], output mean[8], std[8]).  The backward pass is the chain rule
written out; it is pinned by central finite differences in the tests.
"""
import numpy as np

HID, IN, OUT, USED = 256, 4, 8, 6
W1 = 0
B1 = W1 + HID * IN
W2 = B1 + HID
B2 = W2 + HID * HID
W3 = B2 + HID
B3 = W3 + HID * HID
W4 = B3 + HID
B4 = W4 + OUT * HID
NORM = B4 + OUT
SIZE = NORM + 24


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    return dict(W1=P[W1:B1].reshape(HID, IN), b1=P[B1:W2], W2=P[W2:B2].reshape(HID, HID), b2=P[B2:W3],
                W3=P[W3:B3].reshape(HID, HID), b3=P[B3:W4], W4=P[W4:B4].reshape(OUT, HID), b4=P[B4:NORM],
                scale=P[NORM:NORM + 4], shift=P[NORM + 4:NORM + 8], mu=P[NORM + 8:NORM + 16], sd=P[NORM + 16:NORM + 24])


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(P, x):
    """Normalised outputs [rows][8] and the intermediates of the backward pass."""
    p = unpack(P)
    xn = (np.asarray(x, np.float64) - p["shift"]) * p["scale"]
    z1 = xn @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = silu(z3)
    out = h3 @ p["W4"].T + p["b4"]
    return out, dict(xn=xn, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def loss(P, x, y):
    p = unpack(P)
    out, _ = forward(P, x)
    yn = (np.asarray(y, np.float64) - p["mu"][:USED]) / p["sd"][:USED]
    d = out[:, :USED] - yn
    return float((d * d).mean())


def grad(P, x, y):
    """Gradient of loss() with respect to every weight and bias (flat, length NORM)."""
    p = unpack(P)
    out, c = forward(P, x)
    rows = out.shape[0]
    yn = (np.asarray(y, np.float64) - p["mu"][:USED]) / p["sd"][:USED]
    dout = np.zeros_like(out)
    dout[:, :USED] = 2.0 * (out[:, :USED] - yn) / (rows * USED)
    g = np.zeros(NORM)
    g[W4:B4] = (dout.T @ c["h3"]).ravel()
    g[B4:NORM] = dout.sum(0)
    dz3 = (dout @ p["W4"]) * dsilu(c["z3"])
    g[W3:B3] = (dz3.T @ c["h2"]).ravel()
    g[B3:W4] = dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * dsilu(c["z2"])
    g[W2:B2] = (dz2.T @ c["h1"]).ravel()
    g[B2:W3] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * dsilu(c["z1"])
    g[W1:B1] = (dz1.T @ c["xn"]).ravel()
    g[B1:W2] = dz1.sum(0)
    return g


def predict(P, x):
    """Un-normalised predictions [rows][6]: dt, ln r, theta, phi, k^theta, k^r."""
    p = unpack(P)
    out, _ = forward(P, x)
    return out[:, :USED] * p["sd"][:USED] + p["mu"][:USED]


# ---------------------------------------------------------------------------------------
# Crossing network: the same hidden layers with 16 outputs, four per equatorial crossing
# n = 0..3 of the ray (sec. 4.2.1's plane theta = pi/2): a presence logit, ln r_n, the affine
# length since the previous crossing (the first one against the straight line's length to
# the plane) and E_obs/E_em of a Keplerian emitter there.  Flat layout as above with OUT = 16
# and 40 normalisation constants (input scale[4], shift[4], output mean[16], std[16]).
# Loss per row and output, averaged over rows x 16: presence entries (o % 4 == 0, target 0
# or 1) the logistic loss log(1 + e^z) - y z; the others (z - (y - mu)/sigma)^2, or nothing
# where the target is NaN (an absent crossing, or a radius inside the ISCO for the ratio).
# ---------------------------------------------------------------------------------------
XOUT = 16
XW4 = B3 + HID
XB4 = XW4 + XOUT * HID
XNORM = XB4 + XOUT
XSIZE = XNORM + 8 + 2 * XOUT


def x_unpack(P):
    P = np.asarray(P, dtype=np.float64)
    return dict(W1=P[W1:B1].reshape(HID, IN), b1=P[B1:W2], W2=P[W2:B2].reshape(HID, HID), b2=P[B2:W3],
                W3=P[W3:B3].reshape(HID, HID), b3=P[B3:XW4], W4=P[XW4:XB4].reshape(XOUT, HID), b4=P[XB4:XNORM],
                scale=P[XNORM:XNORM + 4], shift=P[XNORM + 4:XNORM + 8], mu=P[XNORM + 8:XNORM + 8 + XOUT],
                sd=P[XNORM + 8 + XOUT:XSIZE])


def x_forward(P, x):
    """Normalised outputs [rows][16] and the intermediates of the backward pass."""
    p = x_unpack(P)
    xn = (np.asarray(x, np.float64) - p["shift"]) * p["scale"]
    z1 = xn @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = silu(z3)
    out = h3 @ p["W4"].T + p["b4"]
    return out, dict(xn=xn, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def _x_terms(p, out, y):
    """Per-entry loss and its derivative with respect to the output."""
    y = np.asarray(y, np.float64)
    pres = (np.arange(XOUT) % 4 == 0)[None, :]
    yn = np.where(pres, y, (y - p["mu"]) / p["sd"])
    valid = ~np.isnan(yn)
    ys = np.where(valid, yn, 0.0)
    sig = 1.0 / (1.0 + np.exp(-out))
    l_pres = np.logaddexp(0.0, out) - ys * out
    l_reg = (out - ys) ** 2
    l = np.where(valid, np.where(pres, l_pres, l_reg), 0.0)
    d = np.where(valid, np.where(pres, sig - ys, 2.0 * (out - ys)), 0.0)
    return l, d


def x_loss(P, x, y):
    p = x_unpack(P)
    out, _ = x_forward(P, x)
    l, _ = _x_terms(p, out, y)
    return float(l.sum() / l.size)


def x_grad(P, x, y):
    """Gradient of x_loss() with respect to every weight and bias (flat, length XNORM)."""
    p = x_unpack(P)
    out, c = x_forward(P, x)
    _, d = _x_terms(p, out, y)
    dout = d / d.size
    g = np.zeros(XNORM)
    g[XW4:XB4] = (dout.T @ c["h3"]).ravel()
    g[XB4:XNORM] = dout.sum(0)
    dz3 = (dout @ p["W4"]) * dsilu(c["z3"])
    g[W3:B3] = (dz3.T @ c["h2"]).ravel()
    g[B3:XW4] = dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * dsilu(c["z2"])
    g[W2:B2] = (dz2.T @ c["h1"]).ravel()
    g[B2:W3] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * dsilu(c["z1"])
    g[W1:B1] = (dz1.T @ c["xn"]).ravel()
    g[B1:W2] = dz1.sum(0)
    return g


def x_predict(P, x):
    """Decoded predictions [rows][16]: per crossing the presence probability, r, the affine
    length term and E_obs/E_em (un-normalised; r = exp of the ln r output)."""
    p = x_unpack(P)
    out, _ = x_forward(P, x)
    v = out * p["sd"] + p["mu"]
    res = v.copy()
    res[:, 0::4] = 1.0 / (1.0 + np.exp(-out[:, 0::4]))
    res[:, 1::4] = np.exp(v[:, 1::4])
    return res
