/*
 * hdfilter.h -- C ABI of the GB300 (sm_103a) fast high-dimensional bilateral /
 * nonlocal-means filter of Nair & Chaudhury, "Fast High-Dimensional Bilateral
 * and Nonlocal Means Filtering" (IEEE TIP; arXiv 1811.02363).
 *
 * What is computed (paper notation):
 *   f : Omega -> R^n      image, n channels          (Eq. (1))
 *   p : Omega -> R^rho    guide, rho dimensions      (Eq. (1))
 *   omega(j) = exp(-|j|^2 / 2 sigma_s^2) on W = [-S, S]^2      (Sec. III)
 *   phi(x)   = exp(-|x|^2 / 2 sigma_r^2)                         (Sec. III)
 *   Brute force:  g(i) = sum_j omega(j) phi(p(i-j)-p(i)) f(i-j) / eta(i)
 *                                                      (Eq. (1)-(2))
 *   Fast filter (Algorithm 1): centres mu_k from bisecting K-means of
 *   {p(i)} (Sec. II-C); A_kl = phi(mu_k - mu_l), b_k(i) = phi(mu_k - p(i))
 *   (Eq. (12)); c(i) = A^+ b(i) (Eq. (11)) or the indicator c(i) = e_s
 *   (Eq. (17)); g_hat = sum_k c_k (omega*(b_k f)) / sum_k c_k (omega*b_k)
 *   (Eq. (15)-(16)).
 *
 * Conventions for every entry point:
 *   - Images are planar float32, (channels, H, W) row-major, contiguous,
 *     pixel i = y*W + x.  Guides are planar (rho, H, W), float32 or bfloat16
 *     (hdf_desc.guide_dtype).  The guide may alias the image (p == f) when
 *     rho == n and the guide is float32 (plain bilateral filter).
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device;
 *     pointers named h_* are HOST pointers.  The caller owns every buffer it
 *     passes; the library never frees or retains them past the call.
 *   - `stream` is a cudaStream_t (0 = legacy default stream).  Device work
 *     is enqueued on it and the call returns without waiting, except where
 *     the comment says it synchronises.
 *   - Window outside the image: neighbours outside Omega are left out of
 *     every sum (zero extension of the convolved images).
 *   - Errors: every call returns an hdf_status; on anything but HDF_OK no
 *     device work was enqueued (argument errors) or the CUDA error is
 *     reported (HDF_ECUDA).  Faults detected on the device (a bounded wait
 *     that gave up, a capacity overflow) are recorded in the handle's device
 *     status word and reported by hdf_get_stats.
 */
#ifndef HDFILTER_H
#define HDFILTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HDF_OK = 0,
  HDF_EINVAL = 1,        /* bad argument: shape, sigma <= 0, K out of range, NULL */
  HDF_ENOMEM = 2,        /* device allocation failed in hdf_create */
  HDF_ECUDA = 3,         /* a CUDA runtime call failed (see hdf_last_cuda_error) */
  HDF_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
  HDF_EDOMAIN = 5,       /* non-finite value met where the method needs finite data */
  HDF_EUNSUPPORTED = 6   /* valid request the library does not handle (e.g. S > 32) */
} hdf_status;

enum { HDF_GUIDE_F32 = 0, HDF_GUIDE_BF16 = 1 };
enum { HDF_COEF_OPT = 0,        /* c(i) = A^+ b(i), Eq. (11) */
       HDF_COEF_INDICATOR = 1   /* c(i) = e_s, s the nearest centre, Eq. (17) */ };
enum { HDF_SPATIAL_GAUSS = 0,   /* omega(j) = exp(-|j|^2 / 2 sigma_s^2) on W (Sec. III) */
       HDF_SPATIAL_BOX = 1,     /* omega(j) = 1 on W, the kernel Sec. III uses for nonlocal
                                   means; sigma_s only sets S when S = 0 */
       HDF_SPATIAL_YOUNG = 2    /* the Gaussian by Young and van Vliet's recursive filter,
                                   the O(1) convolution Sec. II-C names: causal then
                                   anticausal third-order recursions along rows, then
                                   columns, zero states at the borders; sigma_s >= 0.5, S
                                   unused by the convolutions.  hdf_apply only: the batch,
                                   hdf_apply_static and hdf_backward return
                                   HDF_EUNSUPPORTED; hdf_bruteforce computes the exact
                                   Gaussian it approximates */ };

/* Limits of the library. */
#define HDF_MAX_K 64           /* clusters */
#define HDF_MAX_RHO 64         /* guide dimensions */
#define HDF_MAX_S 32           /* window half-width */
#define HDF_MAX_N 256          /* image channels */

typedef struct {
  int H, W;          /* image size, H, W >= 1 */
  int n;             /* channels of f, 1..HDF_MAX_N */
  int rho;           /* dimensions of the guide p, 1..HDF_MAX_RHO */
  int K;             /* clusters requested, 1..HDF_MAX_K (K_eff <= K after clustering) */
  int S;             /* window half-width; 0 selects ceil(3 sigma_s) (Sec. III) */
  double sigma_s;    /* spatial Gaussian std (pixels), > 0 */
  double sigma_r;    /* range Gaussian std (guide units), > 0 */
  int guide_dtype;   /* HDF_GUIDE_F32 or HDF_GUIDE_BF16 */
  int coef;          /* HDF_COEF_OPT or HDF_COEF_INDICATOR */
  int spatial;       /* HDF_SPATIAL_GAUSS or HDF_SPATIAL_BOX */
} hdf_desc;

typedef struct hdf_handle hdf_handle;

typedef struct {
  int K_eff;             /* number of centres in use */
  int fallback_pixels;   /* pixels of the last hdf_apply that took the denominator guard */
  int device_error;      /* hdf_status recorded on the device (HDF_OK if none) */
  int lloyd_iters_max;   /* largest 2-means iteration count of the last clustering */
  int rounds;            /* parallel split rounds of the last clustering */
  double cluster_error;  /* E_K = sum_k sum_{i in C_k} |p(i) - mu_k|^2 (Theorem 1) */
  int rescued_pixels;    /* pixels of the last hdf_apply recomputed in FP64: their float32
                            denominator sum_k c_k r_k was ill-conditioned (sum_k |c_k| r_k
                            above 64 times its magnitude) or within rounding of the guard's
                            threshold; counted in fallback_pixels when the FP64 guard fires */
  int nlm_sweeps;        /* Jacobi sweeps of the last hdf_nlm_guide's eigendecomposition */
} hdf_stats;

/* Validate `desc`, fill in S if 0, and allocate the device workspace of one
 * filter instance (centres, A^+, per-pixel range maps and coefficients,
 * clustering scratch; with HDF_SPATIAL_YOUNG also K (n+1) H W floats of
 * staged planes).  Synchronous; the only call that allocates.
 * Sec. II (Algorithm 1 needs mu, A^+ and the b_k, c_k maps).
 * Errors: HDF_EINVAL (bad desc), HDF_EUNSUPPORTED (beyond HDF_MAX_*),
 * HDF_ENOMEM. */
hdf_status hdf_create(hdf_handle** out, const hdf_desc* desc);

/* Release everything hdf_create allocated.  Synchronises the device. */
void hdf_destroy(hdf_handle* h);

/* Limit of each device-side wait of hdf_cluster (its grid barriers and the
 * wait of a split's finishing block for the other blocks' partial sums), in
 * seconds, 0..60; the default is 2 s.  A wait that reaches the limit records
 * HDF_ETIMEOUT in the device status word and every block of the launch
 * returns; hdf_get_stats then reports HDF_ETIMEOUT and the centres are not
 * valid.  For failure handling and its tests; not part of the paper's method.
 * Errors: HDF_EINVAL (NULL handle, limit outside 0..60). */
hdf_status hdf_set_wait_limit(hdf_handle* h, double seconds);

/* Stage timing of hdf_apply, for measurement: with on != 0 every following
 * hdf_apply records CUDA events on its stream before the range maps, after
 * them, after the convolution tile kernel and after the last stage
 * (normalisation, guard fix-up, FP64 recomputation).  hdf_get_stage_times
 * then returns the three intervals of the last apply in ms: range maps, tile
 * kernel, the rest (the tile kernel's interval is 0 for the recursive
 * Gaussian).  Creates the events on first use (no device memory); the
 * getter synchronises with the last event.  Not part of the paper's method.
 * Errors: HDF_EINVAL (NULL, or no timed apply yet). */
hdf_status hdf_set_stage_timing(hdf_handle* h, int on);
hdf_status hdf_get_stage_times(hdf_handle* h, float* h_ms, int cap, int* count);

/* The descriptor in effect (S filled in). */
hdf_status hdf_get_desc(const hdf_handle* h, hdf_desc* out);

/* Algorithm 1 "cluster" + "pinv": bisecting K-means of Theta = {p(i)}
 * (Eq. (8), Sec. II-C) on the device, then A (Eq. (12)) and A^+ in FP64.
 * d_p: guide (rho, H, W) in the handle's guide dtype.  Asynchronous, no host
 * synchronisation; K_eff stays on the device (read it with hdf_get_stats or
 * hdf_get_centers). */
hdf_status hdf_cluster(hdf_handle* h, const void* d_p, void* stream);

/* Install K centres given on the host (K x rho float32, row-major) instead of
 * clustering, and compute A and A^+ (Eq. (12), Algorithm 1 "pinv").  K <=
 * desc.K.  Enqueues an async copy from h_mu (the host buffer must stay valid
 * until the stream reaches it; pageable memory makes it synchronous). */
hdf_status hdf_set_centers(hdf_handle* h, const float* h_mu, int K, void* stream);

/* Change the widths of the filter for the following calls: omega of Sec. III
 * takes sigma_s and phi takes sigma_r, while the window half-width S, the
 * centres and every buffer stay.  The spatial taps (or, for the recursive
 * Gaussian, the recursion's coefficients) are taken from sigma_s at each
 * launch; A = [phi(mu_k - mu_l)] of Eq. (12) depends on sigma_r, so when the
 * handle holds centres (after hdf_cluster or hdf_set_centers) A and A^+ are
 * refitted on `stream` (asynchronous).  The clustering does not depend on the
 * widths.  With S frozen, a sigma_s well above S/3 gives the Gaussian of that
 * width truncated to W = [-S, S]^2 (Eq. (1)).  Allocates nothing: with it the
 * gradient of hdf_backward with respect to log sigma_s and log sigma_r can
 * drive an optimisation of the widths on one handle.
 * Errors: HDF_EINVAL (NULL handle; a sigma <= 0 or not finite; sigma_s < 0.5
 * with the recursive Gaussian), HDF_ECUDA. */
hdf_status hdf_set_sigmas(hdf_handle* h, double sigma_s, double sigma_r, void* stream);

/* Copy the centres (K_eff x rho float32) to h_mu (room for desc.K rows) and
 * K_eff to *K_eff.  Synchronises `stream`. */
hdf_status hdf_get_centers(hdf_handle* h, float* h_mu, int* K_eff, void* stream);

/* Copy A^+ (K_eff x K_eff, float64, row-major) to h_out (room for K*K).
 * Synchronises `stream`. */
hdf_status hdf_get_pinv(hdf_handle* h, double* h_out, void* stream);

/* Cluster labels of the last hdf_cluster: d_labels[i] in [0, K_eff), the
 * bisecting partition (Sec. II-C).  d_labels: device int32, H*W. Async. */
hdf_status hdf_get_labels(hdf_handle* h, int32_t* d_labels, void* stream);

/* Algorithm 1 loops "for1"-"for3": range maps b_k, coefficients c, the
 * K(n+1) spatial convolutions and the combine/normalise of Eq. (15)-(16),
 * with the centres installed by hdf_cluster or hdf_set_centers.
 * d_f: (n, H, W) float32; d_p: guide (rho, H, W); d_g: output (n, H, W)
 * float32, must not alias d_f or d_p.  Where sum_k c_k r_k <= 1e-6 max_k r_k
 * the pixel takes the indicator value v_s / r_s (s = nearest centre).  Pixels
 * whose float32 sums are ill-conditioned (see hdf_stats.rescued_pixels) are
 * recomputed in FP64 from Eq. (13)-(16) and their guard decided in FP64
 * (Gaussian and box kernels; the recursive Gaussian keeps float32).
 * Asynchronous, allocates nothing. */
hdf_status hdf_apply(hdf_handle* h, const float* d_f, const void* d_p, float* d_g,
                     void* stream);

/* Gradients of L(g_hat) given G = dL/dg_hat (d_grad_g, (n, H, W)), with the
 * centres and S held fixed:
 *   d_grad_f          (n, H, W): dL/df; when d_p == d_f (guide = image) it
 *                     includes the path through b_k(p) and c(p);
 *   d_grad_log_sigma  2 float64: dL/dlog sigma_s, dL/dlog sigma_r.
 * Convolution outputs are recomputed, not stored.  Requires HDF_COEF_OPT,
 * the Gaussian spatial kernel (HDF_EUNSUPPORTED for the box: no sigma_s
 * derivative) and an A that is full rank under the pinv tolerance (dA^+ of a
 * truncated pseudo-inverse is not defined): HDF_EDOMAIN is recorded otherwise.
 * Asynchronous.  Differentiates Eq. (15)-(16); the paper has no backward pass. */
hdf_status hdf_backward(hdf_handle* h, const float* d_f, const void* d_p,
                        const float* d_grad_g, float* d_grad_f,
                        double* d_grad_log_sigma, void* stream);

/* hdf_backward right after the forward pass: d_g is the output of the last
 * hdf_apply on this handle, made from the same d_f and d_p (the caller
 * vouches for that; their contents must not have changed), and the range
 * maps, coefficients, denominators and guard list that apply left in the
 * handle are used instead of being recomputed (saves the forward pass).  At
 * the pixels that apply recomputed in FP64 the adjoint uses the FP64 value of
 * g_hat.  Errors: HDF_EINVAL when the handle's last state-changing call was
 * not hdf_apply (hdf_backward, hdf_cluster, hdf_set_centers and
 * hdf_set_sigmas each end that state), plus those of hdf_backward. */
hdf_status hdf_backward_after_apply(hdf_handle* h, const float* d_f, const void* d_p,
                                    const float* d_g, const float* d_grad_g, float* d_grad_f,
                                    double* d_grad_log_sigma, void* stream);

/* hdf_apply for callers that cannot allocate device memory: a framework or
 * plug-in host that owns all device memory through its own pool and forbids
 * foreign allocations, or a latency-critical path where a cudaMalloc/cudaFree
 * pair (which can synchronise the device) would stall.  Same result as
 * hdf_create + hdf_set_centers + hdf_apply, but no handle: the scratch it
 * needs lives in one 32 MiB static device array that the library holds on
 * every GPU where it is loaded, until the process exits.
 * The paper has no counterpart of this call.
 *   desc: filter description (desc->K is ignored; K is the argument);
 *         checked exactly as hdf_create checks it (HDF_EINVAL /
 *         HDF_EUNSUPPORTED before anything is enqueued).
 *   d_mu: device float32 centres, K x rho row-major (caller-owned, read only).
 *   d_f, d_p, d_g: as in hdf_apply.
 * A call needs about K*K*12 + H*W*(8*K + 17) bytes of that array; larger
 * requests return HDF_EUNSUPPORTED without enqueuing anything (e.g. K = 32 at
 * 256 x 256 fits, K = 32 at 512 x 512 does not).  No cudaMalloc, cudaFree or
 * allocating library call is made.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the
 * array and it keeps the last call's contents: calls whose GPU work overlaps
 * (other streams, other host threads) race on it and must be serialised.
 * No device-side status is reported (the guard count of Eq. (15)-(16), a
 * truncated pseudo-inverse of A): there is no handle to read it from.
 * HDF_SPATIAL_YOUNG returns HDF_EUNSUPPORTED.  Asynchronous on `stream`. */
hdf_status hdf_apply_static(const hdf_desc* desc, const float* d_mu, int K, const float* d_f,
                            const void* d_p, float* d_g, void* stream);

/* Guide for nonlocal means (Sec. I-A; PCA-NLM, Sec. III-C): the patch x patch
 * neighbourhood of every channel around each pixel (borders mirrored without
 * repeating the edge pixel) is reduced by PCA -- mean patch subtracted,
 * covariance over all pixels, projection on the desc.rho eigenvectors of
 * largest eigenvalue (FP64 eigendecomposition on the device).
 *   d_f: image (desc.n, H, W) float32;  d_p: output guide (desc.rho, H, W)
 *   float32, usable as the guide of hdf_cluster / hdf_apply.
 * Eigenvector signs are arbitrary (the filter only uses distances).  Limits:
 * odd patch, desc.n * patch^2 <= 96, desc.n <= 4, H, W > patch/2; otherwise
 * HDF_EUNSUPPORTED / HDF_EINVAL.  Asynchronous, allocates nothing. */
hdf_status hdf_nlm_guide(hdf_handle* h, const float* d_f, int patch, float* d_p, void* stream);

/* Guide for an anisotropic range kernel (Sec. III-E: separate widths for the
 * low-light and the infrared dimensions of a nonlocal-means guide):
 * d_out[d] = d_p[d] / sigma_r[d] for each of the rho planes.  The
 * anisotropic Gaussian phi(x) = exp(-sum_d x_d^2 / (2 sigma_r[d]^2)) of p is
 * the isotropic Gaussian of unit width of this scaled guide, so hdf_create /
 * hdf_cluster / hdf_apply / hdf_bruteforce / the batch with sigma_r = 1 and
 * the scaled guide filter with the anisotropic kernel (the clustering then
 * runs in the kernel's metric; centres come out in scaled units).
 *   d_p: guide (rho, H, W) float32 or bfloat16 (guide_dtype);
 *   h_sigma_r: host, rho widths > 0;  d_out: (rho, H, W) float32, may equal
 *   d_p for a float32 guide.
 * Asynchronous, allocates nothing.  Errors: HDF_EINVAL (NULL, width <= 0 or
 * not finite, bad dtype), HDF_EUNSUPPORTED (rho > HDF_MAX_RHO). */
hdf_status hdf_scale_guide(const void* d_p, int guide_dtype, int rho, int H, int W,
                           const double* h_sigma_r, float* d_out, void* stream);

/* Brute-force filter, Eq. (1)-(2), by direct summation over the window.
 * Same layouts as hdf_apply.  Asynchronous, allocates nothing. */
hdf_status hdf_bruteforce(const hdf_desc* desc, const float* d_f, const void* d_p,
                          float* d_g, void* stream);

/* Phase trace of the last hdf_cluster: up to `cap` events, each two int64
 * (phase id, device globaltimer in ns) recorded by block 0 of the clustering
 * kernel (at most 2048).  Phase ids at the grid barriers: 1 root sums, 2
 * distance and farthest-point pass, 4 root node, 5 Lloyd iteration, 6
 * partition count, 7 partition scatter, 8 children written; between them:
 * 9 end of block 0's Lloyd pass, 11 Lloyd state reloaded, 12-14 block 0
 * finishing a split (all partial sums arrived, reduced, update published),
 * 15 round set-up done, 16 end of block 0's distance pass.
 * paper_1811_02363_gb300.cluster_trace prints the per-phase breakdown.
 * h_events: host, room for 2*cap int64.  *count = events written.
 * Synchronises `stream`.  Tracing support; not part of the paper's method. */
hdf_status hdf_get_trace(hdf_handle* h, int64_t* h_events, int cap, int* count, void* stream);

/* Statistics and the device status word (see hdf_stats).  Synchronises
 * `stream`.  Returns the recorded device error, if any. */
hdf_status hdf_get_stats(hdf_handle* h, hdf_stats* out, void* stream);

/* ------------------------------------------------------------------------
 * Batches.  Many images of different sizes, channel counts, centre counts
 * and sigmas go through Algorithm 1 together, each stage one launch for the
 * whole batch: the clustering of every guide in one cooperative launch (the
 * grid split into groups of blocks, one group per image, sized by the
 * image's work), one fit launch, one range-map launch, ONE persistent launch
 * of the fused convolution/combine tiles of all images (a work list of
 * (image, tile, plane chunk) items, largest first, taken from a global
 * counter), and one normalisation launch.  The whole run can be captured in
 * a CUDA graph and replayed.  Tile shapes (planes per item, tile height) are
 * chosen per (window bucket, plane count) by hdf_batch_tune, which times the
 * candidates on the bound images.  This is an engineering extension: the
 * paper filters one image at a time.
 * ---------------------------------------------------------------------- */
typedef struct hdf_batch hdf_batch;

enum {
  HDF_BATCH_GRAPH = 1,          /* capture the run into a CUDA graph on first use, then replay */
  HDF_BATCH_TIMED = 2,          /* run without a graph, events between stages (get_times) */
  HDF_BATCH_SKIP_CLUSTER = 4    /* keep every image's centres and A^+ (no clustering, no fit) */
};

typedef struct {
  int SB;        /* compiled window bucket (half-width >= S); 0 marks a clustering-plan trial */
  int planes;    /* n + 1 planes per centre; for SB == 0 the number of clustering groups
                    (0: one group per image) */
  int P, TY;     /* planes per work item, tile height (tile width 32); for SB == 0, P is the
                    blocks per group (0: sized per image) and TY is 0 */
  float ms;      /* best time of the persistent launch over the images of this key (for
                    SB == 0: the clustering launch of the whole batch) */
  int chosen;    /* 1 for the shape (plan) kept */
} hdf_tile_trial;

typedef struct {
  int count;               /* images */
  int graph_state;         /* 0 none yet, 1 captured and replayed, -1 capture failed (eager) */
  int launches_per_run;    /* kernel launches of one run */
  int nitems;              /* work items of the persistent tile launch */
  int ngroups;             /* block groups of the clustering launch */
  int grid_cluster;        /* blocks of the clustering launch */
  int grid_tile;           /* blocks of the persistent tile launch */
  size_t smem_tile;        /* dynamic shared memory of the tile launch, bytes */
  size_t device_bytes;     /* device memory the batch owns */
} hdf_batch_info;

/* Validate `count` descriptors (S filled in when 0), plan the clustering
 * groups (one block group per image while each gets at least 19 blocks,
 * else four equal groups that take their images in turn; hdf_batch_tune
 * times the alternatives) and the default tile shapes, and allocate every
 * workspace in one device arena.  descs[i].guide_dtype selects the guide
 * storage of image i:
 * with HDF_GUIDE_BF16 and a NULL guide at bind time, the run converts the
 * image into a bfloat16 guide it owns (guide = image, rho == n).
 * Synchronous; the only batch call that allocates device memory. */
hdf_status hdf_batch_create(hdf_batch** out, int count, const hdf_desc* descs);

/* Release the batch (synchronises the device). */
void hdf_batch_destroy(hdf_batch* b);

/* Bind the caller's device buffers: d_f[i] image (n, H, W) float32;
 * d_p[i] guide (rho, H, W) in descs[i].guide_dtype, or NULL for guide =
 * image (rho == n; bfloat16 storage made by the run when the dtype is
 * HDF_GUIDE_BF16); d_g[i] output (n, H, W), not aliasing d_f[i] / d_p[i].
 * Host arrays of `count` device pointers.  Writes the device tables
 * (synchronous) and drops a captured graph. */
hdf_status hdf_batch_bind(hdf_batch* b, const float* const* d_f, const void* const* d_p,
                          float* const* d_g);

/* Install K centres for image i (host, K x rho float32) and compute its A^+;
 * image i is then not clustered by hdf_batch_run.  Synchronous. */
hdf_status hdf_batch_set_centers(hdf_batch* b, int i, const float* h_mu, int K);

/* One pass of the method over every bound image.  flags: HDF_BATCH_*.
 * Asynchronous on `stream` (a graph capture, on first use, runs on the host
 * and launches nothing until the replay).  Device faults (a bounded wait that
 * gave up) are recorded per image: hdf_batch_get_stats. */
hdf_status hdf_batch_run(hdf_batch* b, int flags, void* stream);

/* Autotuner: run the batch once; time the clustering launch of the batch
 * under each clustering plan (one block group per image sized by its work,
 * or M = 1, 2, 4, ... equal groups that take their images one after the
 * other) and keep the fastest; then for every (window bucket, plane count)
 * present time each compiled tile shape that fits in shared memory on the
 * persistent launch restricted to those images (best of `reps` runs, CUDA
 * events) and keep the fastest.  Synchronous; drops a captured graph. */
hdf_status hdf_batch_tune(hdf_batch* b, int reps, void* stream);

/* Trials of the last hdf_batch_tune (up to cap); *count = trials. */
hdf_status hdf_batch_get_tuning(hdf_batch* b, hdf_tile_trial* out, int cap, int* count);

/* Force the tile shape of every image of (SB, planes), e.g. from a saved
 * tuning.  HDF_EINVAL if the shape is not a compiled one or does not fit. */
hdf_status hdf_batch_set_shape(hdf_batch* b, int SB, int planes, int P, int TY);

/* Stage times (ms) of the last HDF_BATCH_TIMED run, in order: reset,
 * bfloat16 guides, clustering, fit, range maps, persistent tiles,
 * normalisation.  Synchronises.  *count = stages written (<= cap). */
hdf_status hdf_batch_get_times(hdf_batch* b, float* h_ms, int cap, int* count);

/* Centres of image i (room for descs[i].K x rho floats) and K_eff.  Synchronises. */
hdf_status hdf_batch_get_centers(hdf_batch* b, int i, float* h_mu, int* K_eff);

/* Statistics of image i (as hdf_get_stats).  Synchronises. */
hdf_status hdf_batch_get_stats(hdf_batch* b, int i, hdf_stats* out);

/* Plan and state of the batch. */
hdf_status hdf_batch_get_info(hdf_batch* b, hdf_batch_info* out);

/* Measured peak rates of this device's FP32 and FP64 FMA pipes (FLOP/s,
 * FMA = 2 FLOP), in TFLOP/s: FMA-chain probe kernels over every SM, timed
 * with CUDA events on `stream` (best of three launches after a warm-up).
 * The denominators of the FP32-bound kernels' roofline fractions.
 * Synchronises `stream`.  Measurement support; not part of the paper's
 * method.  Errors: HDF_EINVAL (NULL output), HDF_ECUDA. */
hdf_status hdf_probe_peaks(double* fp32_tflops, double* fp64_tflops, void* stream);

/* Human-readable name of a status code. */
const char* hdf_status_string(hdf_status s);

/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char* hdf_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HDFILTER_H */
