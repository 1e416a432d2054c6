"""Pins of the FP64 network oracle used to check the library's training kernels: the
chain-rule gradient equals central finite differences of the loss.  CPU only."""
import numpy as np

from oracle import mlp


def _random_params(rng):
    P = np.zeros(mlp.SIZE)
    P[: mlp.NORM] = rng.normal(0, 0.2, mlp.NORM)
    P[mlp.NORM:mlp.NORM + 4] = [0.05, 0.05, 2.0, 0.025]
    P[mlp.NORM + 4:mlp.NORM + 8] = [0.0, 0.0, 0.5, 45.0]
    P[mlp.NORM + 8:mlp.NORM + 16] = rng.normal(0, 1, 8)
    P[mlp.NORM + 16:mlp.NORM + 24] = rng.uniform(0.5, 2.0, 8)
    return P


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    P = _random_params(rng)
    x = np.stack([rng.uniform(-20, 20, 16), rng.uniform(-20, 20, 16), rng.uniform(0, 1, 16), rng.uniform(5, 85, 16)], 1)
    y = rng.normal(0, 1, (16, 6))
    g = mlp.grad(P, x, y)
    idx = np.concatenate([rng.choice(np.arange(a, b), 6, replace=False) for a, b in
                          [(mlp.W1, mlp.B1), (mlp.B1, mlp.W2), (mlp.W2, mlp.B2), (mlp.B2, mlp.W3), (mlp.W3, mlp.B3),
                           (mlp.B3, mlp.W4), (mlp.W4, mlp.B4), (mlp.B4, mlp.NORM)]])
    for i in idx:
        h = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (mlp.loss(Pp, x, y) - mlp.loss(Pm, x, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_silu_derivative_and_unused_outputs():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    assert np.allclose(mlp.dsilu(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), atol=1e-8)
    rng = np.random.default_rng(5)
    P = _random_params(rng)
    x = rng.uniform(-1, 1, (8, 4))
    g = mlp.grad(P, x, rng.normal(0, 1, (8, 6)))
    # outputs 6 and 7 carry no loss: their output weights and biases get zero gradient
    W4 = g[mlp.W4:mlp.B4].reshape(8, 256)
    assert np.all(W4[6:] == 0) and np.all(g[mlp.B4 + 6:mlp.NORM] == 0)


def _x_params(rng):
    P = np.zeros(mlp.XSIZE)
    P[: mlp.XNORM] = rng.normal(0, 0.2, mlp.XNORM)
    P[mlp.XNORM:mlp.XNORM + 4] = [0.05, 0.05, 2.0, 0.025]
    P[mlp.XNORM + 4:mlp.XNORM + 8] = [0.0, 0.0, 0.5, 45.0]
    P[mlp.XNORM + 8:mlp.XNORM + 24] = rng.normal(0, 1, 16)
    P[mlp.XNORM + 24:mlp.XNORM + 40] = rng.uniform(0.5, 2.0, 16)
    return P


def _x_targets(rng, rows):
    """Crossing targets with the structure of the generator's: presence 1 for a prefix of the
    four crossings, NaN for the absent ones' regression entries and some ratios."""
    y = rng.normal(0, 1, (rows, 16))
    nx = rng.integers(0, 5, rows)
    for m in range(rows):
        for n in range(4):
            y[m, 4 * n] = 1.0 if n < nx[m] else 0.0
            if n >= nx[m]:
                y[m, 4 * n + 1:4 * n + 4] = np.nan
            elif rng.uniform() < 0.3:
                y[m, 4 * n + 3] = np.nan
    return y


def test_crossing_gradient_matches_finite_differences():
    """The crossing network's loss (logistic presence terms, masked squared errors): the
    chain-rule gradient against central differences of the loss, in every tensor."""
    rng = np.random.default_rng(14)
    P = _x_params(rng)
    x = np.stack([rng.uniform(-20, 20, 24), rng.uniform(-20, 20, 24), rng.uniform(0, 1, 24), rng.uniform(5, 85, 24)], 1)
    y = _x_targets(rng, 24)
    g = mlp.x_grad(P, x, y)
    idx = np.concatenate([rng.choice(np.arange(a, b), 6, replace=False) for a, b in
                          [(mlp.W1, mlp.B1), (mlp.B1, mlp.W2), (mlp.W2, mlp.B2), (mlp.B2, mlp.W3), (mlp.W3, mlp.B3),
                           (mlp.B3, mlp.XW4), (mlp.XW4, mlp.XB4), (mlp.XB4, mlp.XNORM)]])
    for i in idx:
        h = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (mlp.x_loss(Pp, x, y) - mlp.x_loss(Pm, x, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_crossing_loss_optimum_is_the_masked_mle():
    """With the output weights zero every row predicts the output bias c.  The loss is then
    stationary in c exactly at the maximum-likelihood estimates: for a presence logit the
    log-odds of the fraction of ones, for a regression output the mean of the targets that
    are present (normalised), NaN entries carrying no weight.  The gradient with respect to
    the output bias vanishes there and not at the unmasked mean."""
    rng = np.random.default_rng(15)
    P = _x_params(rng)
    P[mlp.XW4:mlp.XB4] = 0.0
    x = rng.uniform(-1, 1, (40, 4))
    y = _x_targets(rng, 40)
    mu, sd = P[mlp.XNORM + 8:mlp.XNORM + 24], P[mlp.XNORM + 24:mlp.XNORM + 40]
    c = np.zeros(16)
    for o in range(16):
        col = y[:, o]
        if o % 4 == 0:
            f = col.mean()
            c[o] = np.log(f / (1 - f))
        else:
            c[o] = np.nanmean((col - mu[o]) / sd[o])
    P[mlp.XB4:mlp.XNORM] = c
    g = mlp.x_grad(P, x, y)
    assert np.max(np.abs(g[mlp.XB4:mlp.XNORM])) < 1e-14
    # the unmasked mean (NaN read as the normalised zero) is not stationary
    o = 2
    col = np.where(np.isnan(y[:, o]), mu[o], y[:, o])
    P2 = P.copy()
    P2[mlp.XB4 + o] = ((col - mu[o]) / sd[o]).mean()
    assert abs(mlp.x_grad(P2, x, y)[mlp.XB4 + o]) > 1e-4
    # and the decoded prediction inverts the normalisation: r = exp(mu + sd c)
    pr = mlp.x_predict(P, x[:1])
    assert abs(pr[0, 1] - np.exp(mu[1] + sd[1] * c[1])) < 1e-12 * pr[0, 1]
    assert abs(pr[0, 0] - 1 / (1 + np.exp(-c[0]))) < 1e-15
