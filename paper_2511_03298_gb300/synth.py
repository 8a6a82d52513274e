"""Seeded synthetic workloads (inputs only: no step of the search lives here).

These stand in for the paper's datasets (Table 5), which are not available:
  small  : 10k x 128 isotropic Gaussian mixture (100 centres U[-5,5], sigma 1), L2
  sift   : 1M x 128 non-negative integer vectors 0..255 from a 1000-component
           mixture with a skewed per-dimension scale s_t (SIFT1M / BIGANN shape),
           L2: 30 super-centres U[0, 96 s_t], 1000 component centres at
           N(0, (10 s_t)^2) around them, points at N(0, (20 s_t)^2) around
           those, rounded and clipped (many zeros, as in SIFT).  Components
           crowd together unevenly, so list boundaries cut through dense
           regions: the share of queries with 9 of 10 neighbours in their
           first P of 1024 lists grows from ~1/4 at P = 1 to ~3/4 at P = 8,
           as on SIFT1M
  glove  : 1.2M x 100 unit-norm anisotropic mixture, 2000 components with
           power-law weights (GLOVE-100 / TEXT-TO-IMAGE shape), inner product
  deep   : 10M x 96 unit-norm mixture, 10000 components with Zipf(1.1) weights
           (DEEP10M shape), L2 on normalised data
  fashion: 60k x 784 28x28 image-like vectors, integers 0..255 (FASHION-MNIST
           shape, L2): 100 smooth templates (sums of 3-6 Gaussian bumps on the
           inner 24x24 pixels), each image a template times a brightness
           U[0.7, 1.3] plus N(0, 25^2) pixel noise, rounded and clipped; the
           2-pixel border frame is 0 except for stray pixels (probability
           0.002, U{1..40}), like the uniform backgrounds of Sec. 4.3
Queries come from the same mixture with their own seed.  Seeds: base 1000+c,
queries 2000+c, training queries 3000+c, per-query nprobe 4000+c, build
permutation 5000+c (c = config number 1..6).  Both the CUDA library and the
CPU oracle receive these arrays as inputs; this module computes nothing else.
"""
import numpy as np

GENERATOR_VERSION = 3

CONFIGS = {
    1: dict(name="small", n=10_000, d=128, nq=100, L=64, M=64, k=10, R=100, nprobe=8, metric="l2",
            spherical=False),
    2: dict(name="sift", n=1_000_000, d=128, nq=10_000, L=1024, M=64, k=10, R=200, nprobe=32,
            metric="l2", spherical=False),
    3: dict(name="glove", n=1_200_000, d=100, nq=10_000, L=2048, M=50, k=10, R=200, nprobe=32,
            metric="ip", spherical=True),
    4: dict(name="deep", n=10_000_000, d=96, nq=16_384, L=8192, M=48, k=100, R=1000, nprobe=64,
            metric="l2", spherical=True),
    6: dict(name="fashion", n=60_000, d=784, nq=10_000, L=256, M=196, k=10, R=200, nprobe=8,
            metric="l2", spherical=False),
}
NPROBE_GRID = (8, 12, 16, 24, 32, 48, 64, 96, 128)


def _normalise(a):
    return a / np.linalg.norm(a, axis=-1, keepdims=True)


def _mixture_params(cfg):
    rng = np.random.default_rng(1000 + cfg)
    c = CONFIGS[cfg]
    d = c["d"]
    if cfg == 1:
        mu = rng.uniform(-5.0, 5.0, size=(100, d))
        return dict(mu=mu, w=np.full(100, 1 / 100))
    if cfg == 2:
        s = np.exp(rng.normal(0.0, 0.5, size=d))
        sup = rng.uniform(0.0, 1.0, size=(30, d)) * (96.0 * s)
        mu = sup[rng.integers(0, 30, 1000)] + rng.normal(size=(1000, d)) * (10.0 * s)
        return dict(mu=mu, s=s, w=np.full(1000, 1 / 1000))
    if cfg == 3:
        ncomp = 2000
        mu = _normalise(rng.normal(size=(ncomp, d)))
        sig = 0.08 * np.exp(rng.normal(0.0, 0.5, size=(ncomp, d)))
        w = 1.0 / np.arange(1, ncomp + 1)
        return dict(mu=mu, sig=sig, w=w / w.sum())
    if cfg == 4:
        ncomp = 10_000
        mu = _normalise(rng.normal(size=(ncomp, d)))
        w = np.arange(1, ncomp + 1, dtype=np.float64) ** -1.1
        return dict(mu=mu, w=w / w.sum())
    if cfg == 6:
        ncomp = 100
        yy, xx = np.mgrid[0:28, 0:28]
        tpl = np.zeros((ncomp, 28, 28))
        for c_ in range(ncomp):
            for _ in range(rng.integers(3, 7)):
                cy, cx = rng.uniform(5.0, 22.0, size=2)
                sy, sx = rng.uniform(2.0, 6.0, size=2)
                tpl[c_] += rng.uniform(100.0, 255.0) * np.exp(-0.5 * (((yy - cy) / sy) ** 2 + ((xx - cx) / sx) ** 2))
        inner = np.zeros((28, 28), bool)
        inner[2:26, 2:26] = True
        tpl = np.clip(tpl, 0.0, 255.0) * inner
        return dict(mu=tpl.reshape(ncomp, d), inner=inner.reshape(d), w=np.full(ncomp, 1 / ncomp))
    raise ValueError(cfg)


def _draw(cfg, prm, n, rng, chunk=1 << 20):
    d = CONFIGS[cfg]["d"]
    out = np.empty((n, d), np.float32)
    for b in range(0, n, chunk):
        m = min(chunk, n - b)
        comp = rng.choice(len(prm["w"]), size=m, p=prm["w"])
        eps = rng.standard_normal(size=(m, d))
        if cfg == 1:
            x = prm["mu"][comp] + eps
        elif cfg == 2:
            x = np.clip(np.rint(prm["mu"][comp] + 20.0 * prm["s"] * eps), 0, 255)
        elif cfg == 3:
            x = _normalise(prm["mu"][comp] + prm["sig"][comp] * eps)
        elif cfg == 6:
            bright = rng.uniform(0.7, 1.3, size=(m, 1))
            x = np.clip(np.rint(prm["mu"][comp] * bright + 25.0 * eps), 0, 255) * prm["inner"]
            stray = (rng.uniform(size=(m, d)) < 0.002) & ~prm["inner"]
            x = np.where(stray, rng.integers(1, 41, size=(m, d)), x)
        else:
            x = _normalise(prm["mu"][comp] + 0.05 * eps)
        out[b:b + m] = x
    return out


def base(cfg, n=None):
    """Base vectors of config `cfg` (n overrides the size, same mixture)."""
    c = 2 if cfg == 5 else cfg
    prm = _mixture_params(c)
    rng = np.random.default_rng(1000 + c + 100_000)
    return _draw(c, prm, CONFIGS[c]["n"] if n is None else n, rng)


def queries(cfg, nq=None, stream=0):
    """Queries of config `cfg`; stream s > 0 gives an independent batch of the
    same distribution (one per process of a multi-process run)."""
    c = 2 if cfg == 5 else cfg
    prm = _mixture_params(c)
    rng = np.random.default_rng(2000 + c if stream == 0 else [2000 + c, stream])
    return _draw(c, prm, CONFIGS[c]["nq"] if nq is None else nq, rng)


def train_queries(cfg=5, nt=100_000):
    prm = _mixture_params(2)
    rng = np.random.default_rng(3000 + cfg)
    return _draw(2, prm, nt, rng)


def per_query_nprobe(cfg, nq, lo=4, hi=256):
    rng = np.random.default_rng(4000 + cfg)
    return rng.integers(lo, hi + 1, size=nq).astype(np.int32)


def build_perm(cfg, n):
    """Random order of the base rows: the k-means samples are its prefixes."""
    return np.random.default_rng(5000 + cfg).permutation(n).astype(np.int64)


def rng_array(seed, shape, kind="normal"):
    rng = np.random.default_rng(seed)
    if kind == "normal":
        return rng.standard_normal(size=shape).astype(np.float32)
    if kind == "uniform":
        return rng.uniform(size=shape).astype(np.float32)
    raise ValueError(kind)
