"""FP64 CPU oracle for fast high-dimensional bilateral / nonlocal-means filtering
(Nair & Chaudhury, "Fast High-Dimensional Bilateral and Nonlocal Means
Filtering", IEEE TIP, arXiv 1811.02363).

TEST INFRASTRUCTURE.  This module exists only to check the CUDA library: the
tests, the package smoke check and the benchmark's CPU-baseline leg import it.
Nothing on the product path may call it.  It shares no code with the CUDA
path; it takes plain numpy arrays and works in float64 throughout.

Layout convention: an image with n channels is an array (n, H, W); a guide
with rho dimensions is (rho, H, W); pixel i = (y, x) is enumerated in raster
order y * W + x.

Every function states the passage it follows.  Readings of passages the
paper leaves open (boundary handling, window size, tie rules, the pinv
tolerance, the denominator guard, ...) are listed in the module docstring of
each function and mirrored by the CUDA path.

Parity status: every function below is pinned by tests under ``tests/``
(closed forms, invariants, brute force on tiny inputs, library routines in the
special cases where they coincide) except where its docstring says
"parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np

MAX_LLOYD_ITERS = 20          # cap on 2-means iterations per split (reading of Sec. II-C)
GUARD_REL = 1e-6              # denominator guard, relative to max_k r_k(i)


# --------------------------------------------------------------------------
# Kernels (Sec. III, the isotropic Gaussian range and spatial kernels)
# --------------------------------------------------------------------------

def window_halfwidth(sigma_s: float) -> int:
    """S = ceil(3 sigma_s): Sec. III sets the window W = [-S, S]^2 with S = 3
    sigma_s for bilateral filtering; a non-integer 3 sigma_s is rounded up."""
    return int(math.ceil(3.0 * sigma_s))


def spatial_weights_1d(sigma_s: float, S: int, spatial: str = "gauss") -> np.ndarray:
    """omega_1(t) = exp(-t^2 / 2 sigma_s^2) for t = -S..S.  The 2-D spatial
    kernel of Sec. III, omega(j) = exp(-|j|^2 / 2 sigma_s^2), is the outer
    product omega_1(j_1) omega_1(j_2) (unnormalised: the scale cancels in
    Eq. (1)-(2)).  ``spatial='box'``: the box kernel Sec. III uses for
    nonlocal means, omega = 1 on W, i.e. omega_1 = 1 (sigma_s unused)."""
    t = np.arange(-S, S + 1, dtype=np.float64)
    if spatial == "box":
        return np.ones_like(t)
    if spatial != "gauss":
        raise ValueError(spatial)
    return np.exp(-(t * t) / (2.0 * sigma_s * sigma_s))


def spatial_weight(j1, j2, sigma_s: float, spatial: str = "gauss"):
    """omega(j) at offsets j = (j1, j2) inside W: the Gaussian of Sec. III or
    1 for the box kernel (arrays broadcast)."""
    if spatial == "box":
        return np.ones(np.broadcast(j1, j2).shape) if np.ndim(j1) or np.ndim(j2) else 1.0
    if spatial != "gauss":
        raise ValueError(spatial)
    return np.exp(-(np.asarray(j1, dtype=np.float64) ** 2 + np.asarray(j2, dtype=np.float64) ** 2)
                  / (2.0 * sigma_s * sigma_s))


def range_kernel(sq_dist: np.ndarray, sigma_r: float) -> np.ndarray:
    """phi(x) = exp(-|x|^2 / 2 sigma_r^2) evaluated from |x|^2 (Sec. III)."""
    return np.exp(-sq_dist / (2.0 * sigma_r * sigma_r))


def is_anisotropic(sigma_r) -> bool:
    """sigma_r given per guide dimension (a sequence) rather than as one number."""
    return np.ndim(sigma_r) > 0


def range_kernel_diff(diff: np.ndarray, sigma_r, axis: int) -> np.ndarray:
    """phi of the differences `diff`, the guide dimension along `axis`.
    With one sigma_r: the isotropic Gaussian of Sec. III.  With one sigma_r
    per dimension: the anisotropic Gaussian of Sec. III-E (a separate width
    for the low-light and the infrared dimensions of the guide),
      phi(x) = exp(-sum_d x_d^2 / (2 sigma_{r,d}^2))."""
    diff = np.asarray(diff, dtype=np.float64)
    if not is_anisotropic(sigma_r):
        return range_kernel((diff ** 2).sum(axis=axis), sigma_r)
    s = np.asarray(sigma_r, dtype=np.float64)
    ax = axis % diff.ndim
    if s.shape != (diff.shape[ax],):
        raise ValueError("one sigma_r per guide dimension")
    shape = [1] * diff.ndim
    shape[ax] = -1
    return np.exp(-((diff ** 2) / (2.0 * s * s).reshape(shape)).sum(axis=axis))


def scaled_guide(p: np.ndarray, sigma_r) -> np.ndarray:
    """The guide in the units of the anisotropic kernel's exponent: dimension d
    divided by sigma_{r,d}, so that the anisotropic Gaussian of p is the
    isotropic one of unit width of the scaled guide.  Reading (the paper is
    silent): with an anisotropic kernel the clustering of Theta, Sec. II-C,
    runs in these units, the metric the kernel uses (Theorem 1's Lipschitz
    bound holds in it); so does the nearest-centre choice of Eq. (17)."""
    s = np.asarray(sigma_r, dtype=np.float64)
    return np.asarray(p, dtype=np.float64) / s.reshape(-1, *([1] * (np.ndim(p) - 1)))


# --------------------------------------------------------------------------
# Brute force: Eq. (1) and Eq. (2)
# --------------------------------------------------------------------------

def bruteforce(f: np.ndarray, p: np.ndarray, sigma_s: float, sigma_r: float,
               S: int, spatial: str = "gauss") -> np.ndarray:
    """g(i) = sum_{j in W} omega(j) phi(p(i-j) - p(i)) f(i-j) / eta(i), with
    eta(i) the same sum without f (Eq. (1), Eq. (2)); W = [-S, S]^2.

    Boundary reading: neighbours i-j outside the image are left out of both
    sums (the paper is silent).  eta(i) >= omega(0) phi(0) = 1, so the ratio
    is always defined.  The loop runs over the window offsets j; each
    iteration adds that offset's term for every pixel at once."""
    f = np.asarray(f, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    n, H, W = f.shape
    num = np.zeros((n, H, W))
    den = np.zeros((H, W))
    for j1 in range(-S, S + 1):
        for j2 in range(-S, S + 1):
            w = float(spatial_weight(j1, j2, sigma_s, spatial))
            # pixels i = (y, x) whose neighbour i - j = (y - j1, x - j2) is inside
            y0, y1 = max(0, j1), min(H, H + j1)
            x0, x1 = max(0, j2), min(W, W + j2)
            if y0 >= y1 or x0 >= x1:
                continue
            pi = p[:, y0:y1, x0:x1]
            pn = p[:, y0 - j1:y1 - j1, x0 - j2:x1 - j2]
            wt = w * range_kernel_diff(pn - pi, sigma_r, axis=0)
            num[:, y0:y1, x0:x1] += wt * f[:, y0 - j1:y1 - j1, x0 - j2:x1 - j2]
            den[y0:y1, x0:x1] += wt
    return num / den


def bruteforce_at(f: np.ndarray, p: np.ndarray, sigma_s: float, sigma_r: float,
                  S: int, pixels: np.ndarray, spatial: str = "gauss") -> np.ndarray:
    """Eq. (1)-(2) evaluated at the listed pixels only (rows of (y, x)), one
    pixel at a time by a direct sum over its window.  Returns (len, n)."""
    f = np.asarray(f, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    n, H, W = f.shape
    out = np.empty((len(pixels), n))
    for m, (y, x) in enumerate(pixels):
        ya, yb = max(0, y - S), min(H, y + S + 1)
        xa, xb = max(0, x - S), min(W, x + S + 1)
        dy = (y - np.arange(ya, yb, dtype=np.float64))[:, None]
        dx = (x - np.arange(xa, xb, dtype=np.float64))[None, :]
        w = spatial_weight(dy, dx, sigma_s, spatial)
        wt = w * range_kernel_diff(p[:, ya:yb, xa:xb] - p[:, y:y + 1, x:x + 1], sigma_r, axis=0)
        out[m] = (wt * f[:, ya:yb, xa:xb]).sum(axis=(1, 2)) / wt.sum()
    return out


# --------------------------------------------------------------------------
# Clustering the range space Theta: bisecting K-means (Sec. II-C)
# --------------------------------------------------------------------------

def cluster_sse(X: np.ndarray) -> float:
    """Sum of squared distances of the rows of X to their mean; exactly 0
    when all rows coincide (a rounded mean would otherwise leave a spurious
    positive value and make an unsplittable cluster look splittable)."""
    if len(X) == 0 or np.all(X == X[0]):
        return 0.0
    return float(((X - X.mean(axis=0)) ** 2).sum())


def two_means_split(X: np.ndarray, max_iter: int = MAX_LLOYD_ITERS) -> np.ndarray:
    """Split the rows of X into two parts by 2-means (Sec. II-C).

    Initialisation: the paper starts from a pair of points with the largest
    separation; as a reading, take a = the point farthest from the mean and
    b = the point farthest from a (ties -> first row).  Lloyd iterations:
    assign each point to the nearer centre (tie -> centre a), move each centre
    to the mean of its points, stop when no assignment changes or after
    ``max_iter`` assignments; if an assignment would leave a side empty, keep
    the previous one and stop.

    Returns a boolean array: True = second part (centre b)."""
    mean = X.mean(axis=0)
    a = int(np.argmax(((X - mean) ** 2).sum(axis=1)))
    b = int(np.argmax(((X - X[a]) ** 2).sum(axis=1)))
    ca, cb = X[a].copy(), X[b].copy()
    side = None
    for _ in range(max_iter):
        da = ((X - ca) ** 2).sum(axis=1)
        db = ((X - cb) ** 2).sum(axis=1)
        new = db < da
        if side is not None and (new.all() or not new.any()):
            break
        if side is not None and np.array_equal(new, side):
            break
        side = new
        ca = X[~side].mean(axis=0)
        cb = X[side].mean(axis=0)
    return side


def bisecting_kmeans(P: np.ndarray, K: int, max_iter: int = MAX_LLOYD_ITERS):
    """Bisecting K-means of the range set Theta = {p(i)} (Eq. (8), Algorithm 1
    "cluster", Sec. II-C): starting from one cluster, repeatedly split the
    cluster of largest variance into two by 2-means until there are K
    clusters.

    Readings: "largest variance" = largest sum of squared deviations (SSE),
    ties -> lowest cluster index; splitting stops early (K_eff < K) when the
    largest SSE is 0.  Child 1 keeps the parent's index, child 2 takes the next
    free index.  Centres mu_k are the means of the final clusters.

    P: (N, rho) points in raster order.  Returns (mu (K_eff, rho), labels (N,),
    sse (K_eff,))."""
    P = np.asarray(P, dtype=np.float64)
    N = P.shape[0]
    members = [np.arange(N)]
    sse = [cluster_sse(P)]
    while len(members) < K:
        c = int(np.argmax(sse))
        if sse[c] <= 0.0:
            break
        idx = members[c]
        side = two_means_split(P[idx], max_iter)
        members[c] = idx[~side]
        members.append(idx[side])
        sse[c] = cluster_sse(P[members[c]])
        sse.append(cluster_sse(P[members[-1]]))
    labels = np.empty(N, dtype=np.int64)
    for k, m in enumerate(members):
        labels[m] = k
    mu = np.stack([P[m].mean(axis=0) for m in members])
    return mu, labels, np.asarray(sse)


def clustering_error(P: np.ndarray, mu: np.ndarray, labels: np.ndarray) -> float:
    """E_K = sum_k sum_{p(i) in C_k} |p(i) - mu_k|^2 (Theorem 1)."""
    P = np.asarray(P, dtype=np.float64)
    return float(((P - mu[labels]) ** 2).sum())


def nearest_center(p: np.ndarray, mu: np.ndarray, sigma_r=None) -> np.ndarray:
    """s(i) = argmin_k |p(i) - mu_k|^2, ties -> lowest k (the membership
    "p(i) in C_s" of Eq. (17), read as the Voronoi cell of mu_s); with an
    anisotropic kernel the distance is taken in its units (scaled_guide).
    Returns (H, W) int."""
    p = np.asarray(p, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    if is_anisotropic(sigma_r):
        p = scaled_guide(p, sigma_r)
        mu = mu / np.asarray(sigma_r, dtype=np.float64)[None, :]
    d2 = ((p[None, :, :, :] - mu[:, :, None, None]) ** 2).sum(axis=1)
    return np.argmin(d2, axis=0)


# --------------------------------------------------------------------------
# Shiftable approximation: Eq. (9), (11), (12)
# --------------------------------------------------------------------------

def kernel_matrix(mu: np.ndarray, sigma_r: float) -> np.ndarray:
    """A_kl = phi(mu_k - mu_l) (Eq. (12))."""
    mu = np.asarray(mu, dtype=np.float64)
    if is_anisotropic(sigma_r):
        return range_kernel_diff(mu[:, None, :] - mu[None, :, :], sigma_r, axis=2)
    d2 = ((mu[:, None, :] - mu[None, :, :]) ** 2).sum(axis=2)
    return range_kernel(d2, sigma_r)


def pinv_psd(A: np.ndarray) -> np.ndarray:
    """Moore-Penrose pseudo-inverse of the symmetric PSD matrix A (Algorithm 1
    "pinv"; the paper uses MATLAB's pinv, Sec. II-C).

    A = Q diag(lam) Q^T (symmetric eigendecomposition); eigenvalues with
    |lam| <= tol are dropped, tol = max(size(A)) * eps(norm(A)) as in MATLAB's
    documented default, where norm(A) = max |lam| and eps(x) is the spacing of
    doubles at x.  A^+ = Q_kept diag(1/lam_kept) Q_kept^T."""
    A = np.asarray(A, dtype=np.float64)
    lam, Q = np.linalg.eigh(A)
    norm = float(np.abs(lam).max()) if lam.size else 0.0
    tol = A.shape[0] * float(np.spacing(norm))
    keep = np.abs(lam) > tol
    Qk = Q[:, keep]
    return (Qk / lam[keep]) @ Qk.T


def range_maps(p: np.ndarray, mu: np.ndarray, sigma_r: float) -> np.ndarray:
    """b_k(i) = phi(mu_k - p(i)) (Eq. (12)).  Returns (K, H, W)."""
    p = np.asarray(p, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    if is_anisotropic(sigma_r):
        return range_kernel_diff(p[None, :, :, :] - mu[:, :, None, None], sigma_r, axis=1)
    d2 = ((p[None, :, :, :] - mu[:, :, None, None]) ** 2).sum(axis=1)
    return range_kernel(d2, sigma_r)


# --------------------------------------------------------------------------
# Spatial convolution with the truncated Gaussian (the convolutions of
# Algorithm 1 and the definitions after Eq. (16))
# --------------------------------------------------------------------------

def conv_rows(x: np.ndarray, w1: np.ndarray) -> np.ndarray:
    """out[..., y, c] = sum_t w1(t) x[..., y, c - t], t = -S..S, terms with
    c - t outside the image left out (zero extension)."""
    S = (len(w1) - 1) // 2
    Wd = x.shape[-1]
    out = np.zeros_like(x, dtype=np.float64)
    for t in range(-S, S + 1):
        c0, c1 = max(0, t), min(Wd, Wd + t)
        if c0 < c1:
            out[..., c0:c1] += w1[t + S] * x[..., c0 - t:c1 - t]
    return out


def conv_cols(x: np.ndarray, w1: np.ndarray) -> np.ndarray:
    """The same 1-D convolution along the row index (axis -2)."""
    return np.swapaxes(conv_rows(np.swapaxes(x, -1, -2), w1), -1, -2)


def young_coefficients(sigma_s: float):
    """Coefficients of Young and van Vliet's third-order recursive Gaussian
    (Signal Processing 44, 1995), the O(1) convolution the paper uses for its
    Gaussian spatial kernel (Sec. II-C): q from sigma (their Eq. (11b)),
    b0..b3 (Eq. (8c)) and the gain B = 1 - (b1 + b2 + b3) / b0.  Returns
    (B, a1, a2, a3) with a_i = b_i / b0, so that the causal pass is
    w[t] = B x[t] + a1 w[t-1] + a2 w[t-2] + a3 w[t-3].  Defined for
    sigma >= 0.5."""
    s = float(sigma_s)
    if s >= 2.5:
        q = 0.98711 * s - 0.96330
    elif s >= 0.5:
        q = 3.97156 - 4.14554 * math.sqrt(1.0 - 0.26891 * s)
    else:
        raise ValueError("Young's recursive Gaussian needs sigma >= 0.5")
    b0 = 1.57825 + 2.44413 * q + 1.4281 * q * q + 0.422205 * q ** 3
    b1 = 2.44413 * q + 2.85619 * q * q + 1.26661 * q ** 3
    b2 = -(1.4281 * q * q + 1.26661 * q ** 3)
    b3 = 0.422205 * q ** 3
    return 1.0 - (b1 + b2 + b3) / b0, b1 / b0, b2 / b0, b3 / b0


def young_1d(x: np.ndarray, sigma_s: float, axis: int = -1) -> np.ndarray:
    """The recursive Gaussian along one axis: the causal pass from the first
    sample (zero state before it), then the anticausal pass over its output
    from the last sample (zero state after it):
      w[t] = B x[t] + a1 w[t-1] + a2 w[t-2] + a3 w[t-3],
      y[t] = B w[t] + a1 y[t+1] + a2 y[t+2] + a3 y[t+3].
    Reading: the paper is silent on the boundary; zero states match the zero
    extension used everywhere else.  scipy's lfilter runs each pass (a
    library primitive; the tests pin it against a literal loop)."""
    from scipy.signal import lfilter
    B, a1, a2, a3 = young_coefficients(sigma_s)
    num, den = [B], [1.0, -a1, -a2, -a3]
    x = np.asarray(x, dtype=np.float64)
    w = lfilter(num, den, x, axis=axis)
    y = lfilter(num, den, np.flip(w, axis=axis), axis=axis)
    return np.flip(y, axis=axis)


def spatial_conv(x: np.ndarray, sigma_s: float, S: int, spatial: str = "gauss") -> np.ndarray:
    """(omega * x)(i) = sum_{j in W} omega(j) x(i - j) over the window
    W = [-S, S]^2, zero extension outside the image.  omega factorises, so
    the 2-D sum is done as a row pass followed by a column pass; the tests
    pin this against the direct 2-D sum.  ``spatial='young'``: the Gaussian
    convolution by Young's recursion instead (rows, then columns; S unused),
    the paper's O(1) method -- an approximation of a normalised Gaussian of
    standard deviation sigma_s over the whole image."""
    if spatial == "young":
        return young_1d(young_1d(np.asarray(x, dtype=np.float64), sigma_s, axis=-1),
                        sigma_s, axis=-2)
    w1 = spatial_weights_1d(sigma_s, S, spatial)
    return conv_cols(conv_rows(np.asarray(x, dtype=np.float64), w1), w1)


def spatial_conv_direct(x: np.ndarray, sigma_s: float, S: int,
                        spatial: str = "gauss") -> np.ndarray:
    """Direct 2-D form of ``spatial_conv`` (small inputs)."""
    x = np.asarray(x, dtype=np.float64)
    H, Wd = x.shape[-2:]
    out = np.zeros_like(x)
    for j1 in range(-S, S + 1):
        for j2 in range(-S, S + 1):
            w = float(spatial_weight(j1, j2, sigma_s, spatial))
            y0, y1 = max(0, j1), min(H, H + j1)
            x0, x1 = max(0, j2), min(Wd, Wd + j2)
            if y0 < y1 and x0 < x1:
                out[..., y0:y1, x0:x1] += w * x[..., y0 - j1:y1 - j1, x0 - j2:x1 - j2]
    return out


# --------------------------------------------------------------------------
# Algorithm 1: the fast filter, Eq. (15)-(16)
# --------------------------------------------------------------------------

def fast_filter(f: np.ndarray, p: np.ndarray, mu: np.ndarray, sigma_s: float,
                sigma_r: float, S: int, variant: str = "opt",
                guard: bool = True, return_stats: bool = False, spatial: str = "gauss"):
    """Algorithm 1 with given centres mu (K, rho):

      A (Eq. (12)) and its pseudo-inverse;
      for every pixel: b_k(i) = phi(mu_k - p(i)), u_k(i) = b_k(i) f(i);
      c(i) = A^+ b(i)                         (Eq. (11), ``variant='opt'``)
        or c(i) = e_s, s the nearest centre  (Eq. (17), ``variant='indicator'``)
        or the per-pixel least-squares fit   (Eq. (LS), ``variant='ls'``, see
           ``ls_coefficients``; small images only);
      v = sum_k c_k (omega * u_k), r = sum_k c_k (omega * b_k);
      g_hat = v / r                          (Eq. (15)-(16)).

    Guard (reading; the paper is silent on a vanishing denominator, which can
    occur because c_k may be negative): where r(i) <= 1e-6 max_k (omega*b_k)(i)
    the pixel falls back to the indicator value v_s(i)/r_s(i) (Eq. (18)) with s
    the nearest centre, and to f(i) if r_s(i) is 0 as well.

    ``spatial``: 'gauss' (Sec. III's Gaussian omega), 'box' (omega = 1 on
    W, Sec. III's kernel for nonlocal means) or 'young' (the Gaussian by
    Young's recursion, Sec. II-C's O(1) convolution; S unused).
    Returns g_hat (n, H, W) [, dict(fallback=count)]."""
    f = np.asarray(f, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    n, H, W = f.shape
    K = mu.shape[0]
    A = kernel_matrix(mu, sigma_r)
    A_pinv = pinv_psd(A)
    B = range_maps(p, mu, sigma_r)                                   # (K, H, W)
    s = nearest_center(p, mu, sigma_r)
    if variant == "opt":
        C = np.einsum("kl,lhw->khw", A_pinv, B)
    elif variant == "indicator":
        C = (np.arange(K)[:, None, None] == s[None]).astype(np.float64)
    elif variant == "ls":
        C = ls_coefficients(p, mu, sigma_r, S)
    else:
        raise ValueError(variant)
    v = np.zeros((n, H, W))
    r = np.zeros((H, W))
    r_abs = np.zeros((H, W))          # sum_k |c_k| r_k: the scale of the denominator's rounding
    r_max = np.zeros((H, W))
    v_s = np.zeros((n, H, W))
    r_s = np.zeros((H, W))
    for k in range(K):
        vk = spatial_conv(B[k][None] * f, sigma_s, S, spatial)      # omega * u_k
        rk = spatial_conv(B[k], sigma_s, S, spatial)                # omega * b_k
        v += C[k] * vk
        r += C[k] * rk
        r_abs += np.abs(C[k]) * rk
        np.maximum(r_max, rk, out=r_max)
        sel = s == k
        v_s[:, sel] = vk[:, sel]
        r_s[sel] = rk[sel]
    fallback = (r <= GUARD_REL * r_max) if guard else np.zeros((H, W), dtype=bool)
    safe_r = np.where(fallback, 1.0, r)
    g = v / safe_r
    if fallback.any():
        ind = np.where(r_s > 0, v_s / np.where(r_s > 0, r_s, 1.0), f)
        g = np.where(fallback[None], ind, g)
    if return_stats:
        return g, dict(fallback=int(fallback.sum()), A=A, A_pinv=A_pinv,
                       fallback_mask=fallback, den=r, den_abs=r_abs, r_max=r_max)
    return g


def ls_coefficients(p: np.ndarray, mu: np.ndarray, sigma_r: float, S: int) -> np.ndarray:
    """The coefficients of the per-pixel least-squares problem (LS) of Sec. II:
    c(i) minimises sum_{x in Theta_i} (phi(x - p(i)) - sum_k c_k phi(x - mu_k))^2
    over Theta_i = {p(i - j) : j in W}, the guide values of i's window.

    Readings: Theta_i is taken with multiplicity (one term per window
    position, positions outside the image left out, as in the sums of
    Eq. (1)-(2)); where the problem has several minimisers the minimum-norm
    one is taken (numpy's SVD least squares).  One solve per pixel: the paper
    calls this impractically slow and keeps it only to compare with Eq. (11)
    (its Fig. 6); it is here for that comparison on small images.
    Returns C (K, H, W)."""
    if is_anisotropic(sigma_r):
        raise ValueError("the least-squares coefficients are written for the isotropic kernel")
    p = np.asarray(p, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    rho, H, W = p.shape
    K = mu.shape[0]
    C = np.empty((K, H, W))
    for y in range(H):
        for x in range(W):
            ya, yb = max(0, y - S), min(H, y + S + 1)
            xa, xb = max(0, x - S), min(W, x + S + 1)
            theta = p[:, ya:yb, xa:xb].reshape(rho, -1).T                  # (|Theta_i|, rho)
            M = range_kernel(((theta[:, None, :] - mu[None]) ** 2).sum(axis=2), sigma_r)
            t = range_kernel(((theta - p[:, y, x][None]) ** 2).sum(axis=1), sigma_r)
            C[:, y, x] = np.linalg.lstsq(M, t, rcond=None)[0]
    return C


def fast_filter_at(f: np.ndarray, p: np.ndarray, mu: np.ndarray, sigma_s: float,
                   sigma_r: float, S: int, pixels: np.ndarray,
                   spatial: str = "gauss") -> np.ndarray:
    """Eq. (15)-(16) at the listed pixels only, with v_k(i) and r_k(i) taken
    straight from their definitions Eq. (13)-(14) as sums over the window
    (one pixel at a time).  Same guard as ``fast_filter``.  Returns (len, n)."""
    f = np.asarray(f, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    n, H, W = f.shape
    A_pinv = pinv_psd(kernel_matrix(mu, sigma_r))
    out = np.empty((len(pixels), n))
    for m, (y, x) in enumerate(pixels):
        ya, yb = max(0, y - S), min(H, y + S + 1)
        xa, xb = max(0, x - S), min(W, x + S + 1)
        dy = (y - np.arange(ya, yb, dtype=np.float64))[:, None]
        dx = (x - np.arange(xa, xb, dtype=np.float64))[None, :]
        w = spatial_weight(dy, dx, sigma_s, spatial)
        pw = p[:, ya:yb, xa:xb]
        phi = range_kernel_diff(pw[None] - mu[:, :, None, None], sigma_r, axis=1)   # (K, h, w)
        vk = np.einsum("hw,khw,nhw->kn", w, phi, f[:, ya:yb, xa:xb])  # Eq. (13)
        rk = np.einsum("hw,khw->k", w, phi)                          # Eq. (14)
        b = range_kernel_diff(p[:, y, x][None, :] - mu, sigma_r, axis=1)
        d2i = ((scaled_guide(p[:, y, x], sigma_r)[None, :] - mu / np.asarray(sigma_r))
               ** 2).sum(axis=1) if is_anisotropic(sigma_r) else \
            ((p[:, y, x][None, :] - mu) ** 2).sum(axis=1)
        c = A_pinv @ b
        num = c @ vk
        den = float(c @ rk)
        if den <= GUARD_REL * rk.max():
            s = int(np.argmin(d2i))
            out[m] = vk[s] / rk[s] if rk[s] > 0 else f[:, y, x]
        else:
            out[m] = num / den
    return out


# --------------------------------------------------------------------------
# Nonlocal-means guide: patches reduced by PCA (Sec. I-A, Sec. III-C)
# --------------------------------------------------------------------------

def patch_vectors(f: np.ndarray, patch: int) -> np.ndarray:
    """p(i) = the patch x patch neighbourhood of every channel of f around
    pixel i (Sec. I-A), image borders mirrored without repeating the edge
    pixel.  Returns (n * patch^2, H, W), ordered (channel, dy, dx)."""
    f = np.asarray(f, dtype=np.float64)
    n, H, W = f.shape
    h = patch // 2
    fp = np.pad(f, ((0, 0), (h, h), (h, h)), mode="reflect")
    out = np.empty((n, patch, patch, H, W))
    for a in range(patch):
        for b in range(patch):
            out[:, a, b] = fp[:, a:a + H, b:b + W]
    return out.reshape(n * patch * patch, H, W)


def pca_guide(f: np.ndarray, patch: int = 7, dims: int = 6):
    """PCA-reduced patch guide for nonlocal means (Sec. I-A; Sec. III-C):
    subtract the mean patch, form the covariance of the patch vectors over all
    pixels, project each centred patch onto the ``dims`` eigenvectors of
    largest eigenvalue.  Returns (guide (dims, H, W), basis (dims, D),
    eigenvalues (D,) descending).  Eigenvector signs are arbitrary; the filter
    only uses distances between guide vectors, which do not depend on them."""
    X = patch_vectors(f, patch)
    D, H, W = X.shape
    X = X.reshape(D, H * W)
    mean = X.mean(axis=1, keepdims=True)
    Xc = X - mean
    cov = (Xc @ Xc.T) / (H * W)
    lam, V = np.linalg.eigh(cov)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    basis = V[:, :dims].T
    guide = (basis @ Xc).reshape(dims, H, W)
    return guide, basis, lam


# --------------------------------------------------------------------------
# Accuracy measure: Eq. (21)
# --------------------------------------------------------------------------

def psnr(a: np.ndarray, b: np.ndarray) -> float:
    """PSNR = -10 log10(MSE) with peak 1 and MSE averaged over all n|Omega|
    values (reading of Eq. (21), whose MSE sums channels per pixel)."""
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else -10.0 * math.log10(mse)


def psnr_literal(a: np.ndarray, b: np.ndarray) -> float:
    """Eq. (21) as printed: MSE = |Omega|^-1 sum_i |a(i) - b(i)|^2."""
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    mse = float((d ** 2).sum() / (d.shape[-1] * d.shape[-2]))
    return float("inf") if mse == 0.0 else -10.0 * math.log10(mse)
