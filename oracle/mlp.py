"""FP64 oracle of the learned cost model -- TEST INFRASTRUCTURE ONLY.

The network: x -> relu(x W1 + b1) -> relu(. W2 + b2) -> . W3 + b3 (hidden 64),
loss = mean_i (f(x_i) - y_i)^2.  The gradient is the chain rule written out
layer by layer (backpropagation, Rumelhart, Hinton & Williams 1986); the
update is Adam (Kingma & Ba 2015: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)).  Parameters are one
packed vector: W1 [in][H], b1 [H], W2 [H][H], b2 [H], W3 [H], b3 [1].
"""
import numpy as np

H = 64


def unpack(p, in_dim):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + in_dim * H].reshape(in_dim, H); o += in_dim * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]; o += 1
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def n_params(in_dim):
    return in_dim * H + H + H * H + H + H + 1


def forward(p, X, in_dim):
    W1, b1, W2, b2, W3, b3 = unpack(p, in_dim)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    out = h2 @ W3 + b3
    return out, (X, z1, h1, z2, h2)


def loss_grad(p, X, y, in_dim):
    """(loss, gradient) in float64, by the chain rule."""
    W1, b1, W2, b2, W3, b3 = unpack(p, in_dim)
    out, (X, z1, h1, z2, h2) = forward(p, X, in_dim)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    e = out - y
    loss = float(np.mean(e * e))
    dout = 2.0 * e / n                      # d loss / d out
    gW3 = h2.T @ dout
    gb3 = dout.sum()
    dz2 = np.outer(dout, W3) * (z2 > 0)     # through W3 and the second ReLU
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)           # through W2 and the first ReLU
    gW1 = X.T @ dz1
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def adam_train(p, X, y, in_dim, steps, batch, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam over consecutive minibatches cycling through the samples in order."""
    p = np.array(p, dtype=np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    n = len(y)
    batch = min(batch, n)
    for t in range(1, steps + 1):
        s = ((t - 1) * batch) % n
        c = min(batch, n - s)
        _, g = loss_grad(p, X[s:s + c], y[s:s + c], in_dim)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p
