"""Seeded synthetic workloads (weights, inputs, request streams).

Holds random draws only — none of the method's arithmetic — so that both the
GPU library's tests and the oracle can consume the same inputs.

Recipes (seeds: weights 7751, inputs 2409, keys 1, encryption 2, arrivals 3):
  kan_2_5_1      [2,5,1],  G=5,  k=3, coef N(0,0.1), w_b N(0,0.5), w_s = 1
  kan_4_8_4_1    [4,8,4,1], G=5, k=3, coef N(0,0.1/sqrt(n_i)), w_b N(0,0.5/sqrt(n_i))
  kan_784_64_10  [784,64,10], G=5, k=3, same scaling
  kan_3072_64_10 [3072,64,10], G=10, k=3, same scaling
Inputs: uniform [-1,1]^n_i for the formula models; 28x28 Gaussian-blob
images (1-3 blobs, centre U[4,24]^2, sigma U[2,5] px, amplitude U[128,255],
plus N(0,16^2) noise, clipped to [0,255], rounded, /255) standing in for
MNIST-shaped data; 3x32x32 images N(0.47, 0.25^2) clipped to [0,1]
standing in for CIFAR-10-shaped data.
"""
import numpy as np

SEED_WEIGHTS = 7751
SEED_INPUTS = 2409
SEED_KEYS = 1
SEED_ENC = 2
SEED_ARRIVALS = 3

MODELS = {
    "kan_2_5_1": dict(widths=[2, 5, 1], G=5, k=3, scaled=False),
    "kan_4_8_4_1": dict(widths=[4, 8, 4, 1], G=5, k=3, scaled=True),
    "kan_784_64_10": dict(widths=[784, 64, 10], G=5, k=3, scaled=True),
    "kan_3072_64_10": dict(widths=[3072, 64, 10], G=10, k=3, scaled=True),
}


def make_model(name, seed=SEED_WEIGHTS, widths=None, G=None, k=None):
    spec = dict(MODELS[name]) if name in MODELS else dict(widths=widths, G=G, k=k, scaled=True)
    if widths is not None:
        spec["widths"] = widths
    if G is not None:
        spec["G"] = G
    if k is not None:
        spec["k"] = k
    rng = np.random.default_rng(seed)
    layers = []
    w = spec["widths"]
    for n_in, n_out in zip(w[:-1], w[1:]):
        sc = 1.0 / np.sqrt(n_in) if spec["scaled"] else 1.0
        nb = spec["G"] + spec["k"]
        layers.append(dict(
            n_in=n_in, n_out=n_out, G=spec["G"], k=spec["k"], lo=-1.0, hi=1.0,
            coef=rng.normal(0.0, 0.1 * sc, size=(n_out, n_in, nb)),
            w_s=np.ones((n_out, n_in)),
            w_b=rng.normal(0.0, 0.5 * sc, size=(n_out, n_in)),
        ))
    return layers


def uniform_inputs(n, n_in, seed=SEED_INPUTS):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, n_in))


def blob_images(n, seed=SEED_INPUTS):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:28, 0:28].astype(np.float64)
    out = np.zeros((n, 28 * 28))
    for b in range(n):
        img = np.zeros((28, 28))
        for _ in range(rng.integers(1, 4)):
            cy, cx = rng.uniform(4, 24, size=2)
            s = rng.uniform(2, 5)
            amp = rng.uniform(128, 255)
            img += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * s * s))
        img += rng.normal(0.0, 16.0, size=img.shape)
        out[b] = np.rint(np.clip(img, 0, 255)).ravel() / 255.0
    return out


def cifar_like_images(n, seed=SEED_INPUTS):
    rng = np.random.default_rng(seed)
    x = np.clip(rng.normal(0.47, 0.25, size=(n, 32, 32, 3)), 0.0, 1.0)
    return x.reshape(n, -1)  # raster scan (h, w, c)


def uneven_levels(n, top, slack, seed=SEED_INPUTS + 1):
    """Input levels drawn uniformly from [top - slack, top]."""
    return np.random.default_rng(seed).integers(top - slack, top + 1, size=n)


def poisson_arrivals(rate, duration, seed=SEED_ARRIVALS):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return np.array(out)
        out.append(t)
