"""Seeded synthetic inputs for registration problems.

This module is shared by the CUDA path's tests/benchmarks and by the FP64
oracle.  It holds none of the registration method's arithmetic: images are
closed-form functions of the coordinates, velocities are closed-form
trigonometric polynomials, and the reference image is the template evaluated
at displaced coordinates, m_R(x) = m_T(x - v*(x)) (a first-order stand-in for
the flow of v*, computed without any transport solver).

Workloads (stand-ins for the paper's image data, which are not available):
  * ``blobs_pair``: template = sum of 6 periodic Gaussian blobs
    (sigma in [0.3, 0.8], amplitude in [0.3, 1]); velocity divergence-free with
    modes |k| <= 4.
  * ``labels_pair``: smoothed piecewise-constant 4-label images (level sets of
    a low-mode random field, label intensities U[0, 1]), Gaussian noise
    sigma = 0.01, then Gaussian pre-smoothing with width 2 h (Sec. 4 of the
    paper pre-smooths its data); velocity with modes |k| <= 8 and a
    compressible (gradient) part.
  * ``ellipse_labels``: binary label maps of one of ellipses_pair's ellipses for the
    template and the reference (the label-overlap measures);
  * ``ellipses_pair``: "brain-like" nested smoothed ellipses with 5 labels and
    random contrasts in [0.1, 1]; divergence-free velocity with |k| <= 16.
All images are rescaled to [0, 1] (Sec. 4).
"""
import numpy as np

TWO_PI = 2.0 * np.pi


def coords(n1, n2):
    x1 = TWO_PI * np.arange(n1) / n1
    x2 = TWO_PI * np.arange(n2) / n2
    return np.meshgrid(x1, x2, indexing="ij")


def _trig_poly(n1, n2, coef, kmax, d1=0, d2=0):
    """Real part of sum_{k1,k2 in [-kmax,kmax]} coef[k1,k2] (i k1)^d1 (i k2)^d2 e^{i k.x}
    evaluated on the grid by separable products (closed-form derivatives)."""
    ks = np.arange(-kmax, kmax + 1)
    x1 = TWO_PI * np.arange(n1) / n1
    x2 = TWO_PI * np.arange(n2) / n2
    E1 = np.exp(1j * np.outer(x1, ks))
    E2 = np.exp(1j * np.outer(x2, ks))
    C = coef * ((1j * ks[:, None]) ** d1) * ((1j * ks[None, :]) ** d2)
    return np.real(E1 @ C @ E2.T)


def _trig_poly_at(X1, X2, coef, kmax):
    """Same trigonometric polynomial (no derivative) at arbitrary points."""
    ks = np.arange(-kmax, kmax + 1)
    out = np.zeros(X1.shape)
    for a, k1 in enumerate(ks):
        e1 = np.exp(1j * k1 * X1)
        for b, k2 in enumerate(ks):
            c = coef[a, b]
            if c != 0:
                out += np.real(c * e1 * np.exp(1j * k2 * X2))
    return out


def _random_coef(rng, kmax, decay=1.0):
    ks = np.arange(-kmax, kmax + 1)
    K1, K2 = np.meshgrid(ks, ks, indexing="ij")
    kk = K1 ** 2 + K2 ** 2
    coef = (rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape)) / (1.0 + kk) ** decay
    coef[(kk == 0) | (kk > kmax * kmax)] = 0.0
    return coef


def velocity(n1, n2, kmax, vmax, rng, grad_fraction=0.0):
    """Band-limited velocity (2, n1, n2): curl of a random stream function
    (divergence-free), plus optionally the gradient of a random potential
    scaled to ``grad_fraction`` of the divergence-free part's RMS; the sum is
    scaled to max |v| = vmax.  Modes satisfy |k| <= kmax < n/2."""
    if 2 * kmax >= min(n1, n2):
        raise ValueError("kmax must be below the Nyquist wavenumber")
    psi = _random_coef(rng, kmax)
    v = np.stack([_trig_poly(n1, n2, psi, kmax, d2=1), -_trig_poly(n1, n2, psi, kmax, d1=1)])
    if grad_fraction > 0.0:
        phi = _random_coef(rng, kmax)
        u = np.stack([_trig_poly(n1, n2, phi, kmax, d1=1), _trig_poly(n1, n2, phi, kmax, d2=1)])
        rms_v = np.sqrt(np.mean(v ** 2))
        rms_u = np.sqrt(np.mean(u ** 2))
        v = v + grad_fraction * (rms_v / rms_u) * u
    vabs = np.sqrt(v[0] ** 2 + v[1] ** 2).max()
    return v * (vmax / vabs)


def smooth_field(n1, n2, kmax, rng, decay=1.0):
    """Random smooth scalar field with modes |k| <= kmax, unit max-abs."""
    f = _trig_poly(n1, n2, _random_coef(rng, kmax, decay), kmax)
    return f / np.abs(f).max()


def rescale01(m):
    lo, hi = m.min(), m.max()
    return (m - lo) / (hi - lo)


def _wrap(d):
    return np.mod(d + np.pi, TWO_PI) - np.pi


def _blobs(X1, X2, params):
    out = np.zeros(X1.shape)
    for c1, c2, sig, amp in params:
        d2 = _wrap(X1 - c1) ** 2 + _wrap(X2 - c2) ** 2
        out += amp * np.exp(-d2 / (2.0 * sig * sig))
    return out


def blobs_pair(n, seed, vmax=0.5, kmax=4, nblobs=6):
    """(m_T, m_R, v*) on an n x n grid; see module docstring."""
    rng = np.random.default_rng(seed)
    params = [(rng.uniform(0, TWO_PI), rng.uniform(0, TWO_PI), rng.uniform(0.3, 0.8), rng.uniform(0.3, 1.0))
              for _ in range(nblobs)]
    v = velocity(n, n, kmax, vmax, rng)
    X1, X2 = coords(n, n)
    mT = _blobs(X1, X2, params)
    mR = _blobs(X1 - v[0], X2 - v[1], params)
    lo, hi = mT.min(), mT.max()
    return (mT - lo) / (hi - lo), (mR - lo) / (hi - lo), v


def _ellipse_params(rng, nlabels):
    params = []
    c1, c2 = np.pi + rng.normal(0, 0.05 * np.pi), np.pi + rng.normal(0, 0.05 * np.pi)
    a, b = rng.uniform(0.55, 0.7) * np.pi, rng.uniform(0.45, 0.6) * np.pi
    th = rng.uniform(0, np.pi)
    contrasts = rng.uniform(0.1, 1.0, size=nlabels)
    for lab in range(nlabels):
        params.append((c1, c2, a, b, th, contrasts[lab]))
        s = rng.uniform(0.6, 0.8)
        a, b = a * s, b * s
        c1 += rng.normal(0, 0.1 * a)
        c2 += rng.normal(0, 0.1 * b)
        th += rng.normal(0, 0.3)
    return params


def _ellipses(X1, X2, params, width):
    out = np.zeros(X1.shape)
    prev = 0.0
    for c1, c2, a, b, th, c in params:
        d1, d2 = _wrap(X1 - c1), _wrap(X2 - c2)
        p = np.cos(th) * d1 + np.sin(th) * d2
        q = -np.sin(th) * d1 + np.cos(th) * d2
        r = np.sqrt((p / a) ** 2 + (q / b) ** 2)
        ind = 0.5 * (1.0 + np.tanh((1.0 - r) * np.sqrt(a * b) / width))
        out += (c - prev) * ind
        prev = c
    return out


def ellipses_pair(n, seed, vmax, kmax=16, nlabels=5):
    """Nested smoothed ellipses (edge width 2 h); (m_T, m_R, v*)."""
    rng = np.random.default_rng(seed)
    params = _ellipse_params(rng, nlabels)
    v = velocity(n, n, kmax, vmax, rng)
    X1, X2 = coords(n, n)
    width = 2.0 * TWO_PI / n
    mT = _ellipses(X1, X2, params, width)
    mR = _ellipses(X1 - v[0], X2 - v[1], params, width)
    lo, hi = mT.min(), mT.max()
    return (mT - lo) / (hi - lo), (mR - lo) / (hi - lo), v


def ellipse_labels(n, seed, vmax, kmax=16, nlabels=5, label=1):
    """Binary label maps (1 inside, 0 outside) of the pair ellipses_pair(n, seed, vmax, kmax,
    nlabels) draws: the region inside ellipse `label` (0 = the outermost), for the template
    and, at the displaced coordinates x - v*(x), for the reference; (L_T, L_R)."""
    rng = np.random.default_rng(seed)
    params = _ellipse_params(rng, nlabels)
    v = velocity(n, n, kmax, vmax, rng)
    X1, X2 = coords(n, n)

    def inside(Y1, Y2):
        c1, c2, a, b, th, _ = params[label]
        d1, d2 = _wrap(Y1 - c1), _wrap(Y2 - c2)
        p = np.cos(th) * d1 + np.sin(th) * d2
        q = -np.sin(th) * d1 + np.cos(th) * d2
        return ((p / a) ** 2 + (q / b) ** 2 < 1.0).astype(np.float64)

    return inside(X1, X2), inside(X1 - v[0], X2 - v[1])


def gaussian_smooth(f, sigma):
    """Periodic Gaussian filter of width sigma (data pre-smoothing)."""
    n1, n2 = f.shape
    k1 = np.fft.fftfreq(n1, 1.0 / n1)
    k2 = np.fft.rfftfreq(n2, 1.0 / n2)
    K1, K2 = np.meshgrid(k1, k2, indexing="ij")
    return np.fft.irfft2(np.fft.rfft2(f) * np.exp(-0.5 * sigma * sigma * (K1 ** 2 + K2 ** 2)), s=(n1, n2))


def labels_pair(n, seed, vmax=0.8, kmax=8, nlabels=4, noise=0.01, grad_fraction=0.3):
    """Smoothed noisy piecewise-constant label images; (m_T, m_R, v*)."""
    rng = np.random.default_rng(seed)
    kf = 3
    coef = _random_coef(rng, kf)
    intens = rng.uniform(0.0, 1.0, size=nlabels)
    v = velocity(n, n, kmax, vmax, rng, grad_fraction=grad_fraction)
    X1, X2 = coords(n, n)
    fT = _trig_poly(n, n, coef, kf)
    fR = _trig_poly_at(X1 - v[0], X2 - v[1], coef, kf)
    qs = np.quantile(fT, np.linspace(0, 1, nlabels + 1)[1:-1])

    def render(f):
        lab = np.searchsorted(qs, f)
        return intens[lab]

    h = TWO_PI / n
    mT = gaussian_smooth(render(fT) + noise * rng.standard_normal((n, n)), 2.0 * h)
    mR = gaussian_smooth(render(fR) + noise * rng.standard_normal((n, n)), 2.0 * h)
    return rescale01(mT), rescale01(mR), v


def _ellipses_job(job):
    n, seed, vmax = job
    mT, mR, _ = ellipses_pair(n, seed, vmax=vmax, kmax=min(16, n // 4))
    return mT.astype(np.float32), mR.astype(np.float32)


def ellipses_images(jobs, workers=1):
    """[(m_T, m_R)] float32 for jobs [(n, seed, vmax)] (``ellipses_pair`` with
    kmax = min(16, n/4)); workers > 1 uses spawned worker processes, which is safe
    after CUDA has been initialised in the calling process.  The calling script
    must guard its top level with ``if __name__ == "__main__":`` (spawned workers
    import it); a worker that dies raises BrokenProcessPool here instead of being
    replaced."""
    jobs = list(jobs)
    if workers > 1 and len(jobs) > 32:
        import multiprocessing as mp
        import os
        from concurrent.futures import ProcessPoolExecutor
        # one BLAS thread per worker process (the children inherit this environment)
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as pool:
                return list(pool.map(_ellipses_job, jobs, chunksize=8))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    return [_ellipses_job(j) for j in jobs]
