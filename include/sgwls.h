/*
 * sgwls.h -- C ABI of the GB300 SG-WLS library (libsgwls.so).
 *
 * Semi-Global Weighted Least Squares (Liu, Chen, Shen, Liu, Yang, ICCV 2017)
 * smooths an image F under a guidance image G by repeating, T times, a pass
 * along the column direction and a pass along the row direction (Sec. 2.3).
 * Each pass builds, for every centre line k, the (2r+1)-line strip around k
 * in zig-zag order (Sec. 2.1), solves its 1D WLS subsystem A_s u = f exactly
 * (Eq. 5; A_s formed like Eq. 4 with the Eq. 2 guidance weights over the
 * 2r+1 neighbouring entries of the formed vector), writes the solution back
 * into the strip and averages the values each pixel received.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout     planar C x H x W, row-major, contiguous per image; the guidance
 *            is one H x W plane (or guide_channels planes, planar).  Pixel (y, x) of channel c lives at
 *            c*H*W + y*W + x elements from the base pointer.
 * Pointers   image, guidance, output, workspace and saved-estimate pointers
 *            are DEVICE pointers (cudaMalloc / caching-allocator memory of the
 *            current device); parameter structs and image tables are HOST
 *            pointers.  The caller owns every buffer; the library allocates
 *            nothing and keeps no state between calls.
 * Stream     `stream` is a cudaStream_t passed as void* (NULL = legacy
 *            default stream).  Every call is asynchronous on that stream:
 *            results are ready when the stream has reached the call.
 * Aliasing   the output may alias neither the input nor the guidance
 *            (SGWLS_E_INVALID); the guidance may alias the input (guidance =
 *            input, as in the grayscale workloads).
 * Errors     arguments are validated on the host before anything is
 *            launched; a failed validation returns an SGWLS_E_* code and
 *            touches no memory.  A CUDA launch failure returns SGWLS_E_CUDA
 *            (the CUDA error string is kept by sgwls_last_cuda_error()).
 * Precision  all elimination arithmetic is FP32; no FP64 on the GPU.  Every
 *            pivot (in the chunk sweeps, the separator merges and the
 *            reduced chains) is formed as a row's margin plus the magnitudes
 *            of its remaining couplings, a sum of non-negative terms
 *            (Grassmann-Taksar-Heyman elimination of the M-matrix I + lambda
 *            L), so FP32 keeps A_s's identity where lambda w reaches ~1e7.
 *            `storage` selects FP32 or BF16 for the input/output/guidance
 *            buffers, `inter_storage` for the estimates between passes.
 */
#ifndef SGWLS_H
#define SGWLS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SGWLS_OK = 0,
  SGWLS_E_INVALID = -1,     /* a parameter is out of range or a pointer is NULL */
  SGWLS_E_SHAPE = -2,       /* H, W < 2r+1, C < 1, or sizes too large            */
  SGWLS_E_DTYPE = -3,       /* unknown storage type                              */
  SGWLS_E_WORKSPACE = -4,   /* workspace missing or smaller than required        */
  SGWLS_E_CUDA = -5,        /* a CUDA call failed (see sgwls_last_cuda_error)    */
  SGWLS_E_DEVICE_FLAG = -6, /* a kernel's bounded wait gave up (sgwls_device_flag) */
  SGWLS_E_UNSUPPORTED = -7  /* valid request this build does not implement       */
} sgwls_status;

typedef enum { SGWLS_F32 = 0, SGWLS_BF16 = 1 } sgwls_dtype;

/* Eq. 2: the two guidance weights. */
typedef enum { SGWLS_W_EXP = 0, SGWLS_W_FRAC = 1 } sgwls_weight;

/* User constants of the method.  Fill with sgwls_params_default() first.
 *   weight      Eq. 2 form: exp(-|i-j|^2/2 sigma_s^2) exp(-|Gi-Gj|^2/2 sigma_r^2)
 *               or 1/(|i-j|^alpha_s + eps) * 1/(|Gi-Gj|^alpha_r + eps);
 *               |i-j| is the Euclidean distance of the pixel coordinates.
 *   r           neighbourhood radius, (2r+1)x(2r+1) system, 1 <= r <= SGWLS_R_MAX
 *   iters       T, the number of (column pass, row pass) pairs, >= 0 (Sec. 2.3)
 *   step        tau, the sliding step between subsystem centres (Sec. 2.3),
 *               1 <= step <= 2r+1 (the last centre is always included).
 *               step > 1 runs on kept factors (not factor_cache = 2); the
 *               batched, backward and no-allocation entry points return
 *               SGWLS_E_UNSUPPORTED for step > 1
 *   axis_order  0: column direction first (Sec. 2.3), 1: row direction first
 *   refine      0 or 1: one step of iterative refinement of every
 *               subsystem solve, all in FP32: u1 = A~^-1 f, the residual
 *               rho = f - u1 - lambda L u1 with A = I + lambda L applied
 *               without forming its diagonal (the pair weights recomputed
 *               from the guidance), the solve of rho added to u1, then the
 *               averaging (five kernels per pass instead of two; the
 *               workspace grows by two per-entry buffers).  An extra
 *               correction of the FP32 solve; the plain solve's subtraction-
 *               free pivots already keep the frac weights' large-lambda
 *               settings (lambda w ~1e7) within 2e-4 of FP64.  Needs
 *               step = 1 and kept factors (not factor_cache = 2); the
 *               batched, backward and no-allocation entry points return
 *               SGWLS_E_UNSUPPORTED for refine = 1
 *   storage     sgwls_dtype of f, g and u
 *   inter_storage  sgwls_dtype of the estimates between passes
 *   chunk_lines 0: automatic; otherwise the number of lines per chunk of
 *               the parallel subsystem solve (a tuning knob; the result is
 *               the same up to FP32 rounding for every value)
 *   factor_cache  where the second kernel of a forward or adjoint pass
 *               gets the chunk factors (LDL^T rows and forward-substituted
 *               right-hand sides) from: 0 automatic (kept in the workspace
 *               when one pass's factors take at most 4 GiB, otherwise
 *               recomputed), 1 always kept, 2 always recomputed.  Keeping
 *               costs 4 (2r+1)(2r+C') bytes per pixel of workspace (C' =
 *               right-hand sides per group: at most 4 forward; u and v of
 *               up to 3 channels at r = 1, 2 otherwise, in the backward)
 *               and saves the second kernel's weights and factorisation.  A
 *               tuning knob: the results agree up to FP32 rounding.
 *   guide_channels  Cg, the number of guidance planes: 0 or 1 (g is H x W)
 *               or 2 .. SGWLS_GUIDE_MAX (g is Cg x H x W, planar, type
 *               p->storage); |Gi-Gj| in Eq. 2 is then the Euclidean norm of
 *               the difference of the two pixels' guidance vectors (for
 *               example an RGB guidance image).  Cg > 1 runs on kept factors
 *               (not factor_cache = 2); refine = 1 and the batched, backward
 *               and no-allocation entry points return SGWLS_E_UNSUPPORTED
 *               for Cg > 1.
 *   schedule    how a forward pass with kept factors (sliding step 1, no
 *               refinement, one guidance plane) runs: 0 automatic (= 1),
 *               1 two kernels (every chunk's forward sweep, then every
 *               back substitution), 2 one persistent kernel taking both
 *               kinds of work item from a queue, band by band, so that a
 *               band's factors are read back while they are still in L2
 *               (its waits are bounded: see sgwls_device_flag).  Other
 *               passes ignore it.  A tuning knob: both schedules run the
 *               same arithmetic and give identical results.
 *   ring_slots  schedule 2 only: 0 automatic (as many bands of factors as
 *               fit 64 MiB), or the number of band slots (>= 4) of the
 *               factor-store ring; a band reuses a slot once every reader of
 *               the band before it finished.  A tuning knob.
 *   group_warps 0 automatic (up to 8), or 1, 2, 4, 8: the most chunks
 *               (one warp each) a block of the single-image forward and
 *               backward kernels takes.  A tuning knob.
 *   lookahead   schedule 2 only: 0 automatic (about one generation of
 *               resident blocks), else the number of bands between a band's
 *               forward sweeps and the back substitutions that read it in
 *               the work queue (at most ring_slots - 2 with a ring).  A
 *               tuning knob.                                              */
typedef struct {
  int weight;
  float sigma_s, sigma_r;
  float alpha_s, alpha_r, eps;
  int r;
  int iters;
  int step;
  int axis_order;
  int refine;
  int storage;
  int inter_storage;
  int chunk_lines;
  int factor_cache;
  int guide_channels;
  int schedule;
  int ring_slots;
  int group_warps;
  int lookahead;
} sgwls_params;

#define SGWLS_R_MAX 8
#define SGWLS_C_MAX 64
#define SGWLS_GUIDE_MAX 4

/* Defaults: exp weights, sigma_s = 1, sigma_r = 0.1, alpha_s = alpha_r = 1.2,
 * eps = 1e-4 (Sec. 1), r = 1, iters = 1, step = 1, axis_order = 0,
 * refine = 0, FP32 storage, chunk_lines = 0, factor_cache = 0,
 * guide_channels = 1, schedule = 0, ring_slots = 0, group_warps = 0,
 * lookahead = 0.  `p` must not be NULL. */
void sgwls_params_default(sgwls_params* p);

/* Human-readable name of a status code (static string, never NULL). */
const char* sgwls_status_string(sgwls_status s);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* sgwls_last_cuda_error(void);

/* Workspace bytes sgwls_filter needs for an H x W x C image with `p`
 * (0 if the arguments are invalid).  Host-only; launches nothing. */
size_t sgwls_workspace_bytes(int H, int W, int C, const sgwls_params* p);

/* SG-WLS filter of one image (Sec. 2.3; Eqs. 2, 4, 5).
 *   f       device, C x H x W input (storage type p->storage)
 *   g       device, H x W guidance (p->storage), or Cg x H x W with
 *           p->guide_channels = Cg > 1; may equal f when C == Cg
 *   u       device, C x H x W output (p->storage); must not alias f or g
 *   lambda  smoothness weight of Eq. 1 / Eq. 4, >= 0
 *   ws      device workspace of at least sgwls_workspace_bytes(H, W, C, p)
 *           bytes, 256-byte aligned; contents on entry are ignored
 *   saved   device, NULL or 2*iters*C*H*W elements of type p->inter_storage:
 *           if given, the input estimate of pass t (t = 0 .. 2*iters-1) is
 *           written to element offset t*C*H*W (pass 0's input is a copy of
 *           f), the per-pass checkpoints sgwls_filter_backward reads.
 *   stream  cudaStream_t as void*
 * iters == 0 copies f to u. */
sgwls_status sgwls_filter(const void* f, const void* g, void* u, int H, int W, int C,
                          float lambda, const sgwls_params* p, void* ws, size_t ws_bytes,
                          void* saved, void* stream);

/* One pass of Sec. 2.3 along one direction: for every centre line k the
 * neighbourhood construction (Sec. 2.1), the exact solve of its subsystem
 * (Eq. 5), the inverse construction and the averaging; u = pass(f).
 *   direction  0: column direction (centres are columns), 1: row direction
 * f, g, u, lambda, p, ws, ws_bytes, stream as in sgwls_filter (p->iters is
 * ignored except for workspace sizing; f and u use p->storage).  The
 * workspace of sgwls_workspace_bytes(H, W, C, p) suffices. */
sgwls_status sgwls_filter_pass(const void* f, const void* g, void* u, int H, int W, int C,
                               float lambda, const sgwls_params* p, int direction, void* ws,
                               size_t ws_bytes, void* stream);

/* One image of a batched call (all pointers device pointers). */
typedef struct {
  const void* f;   /* C x H x W input (p->storage)                   */
  const void* g;   /* H x W guidance (p->storage)                    */
  void* u;         /* C x H x W output (p->storage), not aliasing f  */
  int H, W, C;     /* any channel count 1 <= C <= SGWLS_C_MAX per image */
  float lambda;    /* per-image lambda >= 0                           */
  void* saved;     /* NULL, or 2*iters*C*H*W elements (p->inter_storage)
                      receiving the input estimate of every pass, as the
                      `saved` argument of sgwls_filter               */
} sgwls_image;

/* Guided sparse interpolation (Sec. 2.3, Eq. 21): the SG-WLS filter applied
 * to the sparse input F and to its index map Hm, and their ratio per pixel,
 *   U(m) = SGWLS(F)(m) / SGWLS(Hm)(m).
 * Both are filtered with the same guidance and parameters; F's channels and
 * Hm are solved as right-hand sides of one factorisation per subsystem
 * (C + 1 <= 4 share every factor).
 *   f     device, C x H x W sparse input (FP32), zero where hmap is zero
 *   hmap  device, H x W index map (FP32): 1 where f holds data, else 0
 *   g     device, H x W guidance (FP32), or Cg x H x W with
 *         p->guide_channels = Cg > 1
 *   u     device, C x H x W output (FP32); a pixel that no data reaches
 *         (filtered index map exactly 0) is 0
 *   ws    device workspace of at least sgwls_interpolate_workspace_bytes
 *         bytes, 256-byte aligned
 * p->storage and p->inter_storage must be SGWLS_F32 (else
 * SGWLS_E_UNSUPPORTED).  Asynchronous on `stream`; u must not alias f or
 * hmap.  Other errors as sgwls_filter. */
size_t sgwls_interpolate_workspace_bytes(int H, int W, int C, const sgwls_params* p);
sgwls_status sgwls_interpolate(const void* f, const void* hmap, const void* g, void* u, int H, int W, int C,
                               float lambda, const sgwls_params* p, void* ws, size_t ws_bytes,
                               void* stream);

/* Workspace bytes sgwls_filter_batched needs for these images (0 if the
 * arguments are invalid).  Host-only; `imgs` is a host array. */
size_t sgwls_batched_workspace_bytes(int B, const sgwls_image* imgs, const sgwls_params* p);

/* SG-WLS filter of B images of uneven sizes and channel counts (Sec. 2.3
 * per image, each with its own lambda, the same r / T / weights).  Every
 * image is split into channel groups of at most four channels (the channels
 * of a group share each subsystem's factorisation); the groups of equal
 * size form one uniform batch, and every pass of a uniform batch runs as one
 * launch per kernel over all its groups (up to 64 per launch; larger
 * batches use several): each block finds its image from the per-image block
 * ranges carried in the kernel arguments, so no descriptor is uploaded and
 * the call can be captured in a CUDA graph.  A batch of RGB and gray images
 * thus takes two launches per kernel per pass.
 *   imgs  host array of B images; ws: workspace of
 *         sgwls_batched_workspace_bytes bytes, 256-byte aligned.
 * The output of an image may alias neither its input nor its guidance. */
sgwls_status sgwls_filter_batched(int B, const sgwls_image* imgs, const sgwls_params* p, void* ws,
                                  size_t ws_bytes, void* stream);

/* Workspace bytes sgwls_filter_backward needs (0 if the arguments are
 * invalid).  Host-only. */
size_t sgwls_backward_workspace_bytes(int H, int W, int C, const sgwls_params* p);

/* Reverse-mode derivative of sgwls_filter (the paper has no backward pass;
 * this is the chain rule through Eqs. 2, 4, 5 and the four steps of
 * Sec. 2.3).  Per pass, walked in reverse order, for every subsystem with
 * u = A_s^-1 f (recomputed from the checkpoint) and v = A_s^-1 ubar, where
 * ubar gathers dLoss/d(pass output) divided by each pixel's subsystem count:
 *   dLoss/d(pass input) = sum over subsystems of v scattered to the pixels;
 *   dLoss/dlambda      += -sum_pairs w_pq (v_p - v_q).(u_p - u_q);
 *   dLoss/dG           += -lambda (v_p - v_q).(u_p - u_q) dw_pq/dG
 * (the dot runs over channels, which share A_s).
 *   grad_u      device FP32 C x H x W, dLoss/du
 *   g           device FP32 H x W guidance used in the forward call
 *   saved       device FP32 2*iters*C*H*W per-pass checkpoints written by
 *               sgwls_filter (p->inter_storage must be SGWLS_F32)
 *   lambda, p   as in the forward call (FP32 storage; frac weights need
 *               alpha_r >= 1, otherwise SGWLS_E_UNSUPPORTED)
 *   grad_f      device FP32 C x H x W output, dLoss/df (may not alias grad_u)
 *   grad_g      device FP32 H x W output, dLoss/dg, or NULL
 *   grad_lambda device pointer to one float, dLoss/dlambda, or NULL
 *   ws          workspace of sgwls_backward_workspace_bytes bytes, 256-byte
 *               aligned
 * Gradients w.r.t. g and lambda are accumulated with floating-point atomics:
 * their last bits depend on the order of accumulation. */
sgwls_status sgwls_filter_backward(const void* grad_u, const void* g, const void* saved, int H, int W, int C,
                                   float lambda, const sgwls_params* p, void* grad_f, void* grad_g,
                                   float* grad_lambda, void* ws, size_t ws_bytes, void* stream);

/* Line relaxation of the 2D WLS model: an opt-in variant, NOT the paper's
 * SG-WLS subsystem (Sec. 2.1 solves the whole (2r+1)-line zig-zag strip).
 * It reads "each pass solves one 1D system per line with the off-line
 * neighbours at their current estimates" as a block-Jacobi iteration on the
 * dense 2D WLS system of Eqs. 1-4 (A = I + lambda L over the (2r+1) x (2r+1)
 * square neighbourhood, Eq. 2 weights): every pass solves, for each row (row
 * direction) or column (column direction),
 *   (1 + lambda sum_{q in N(p)} w_pq) u_p - lambda sum_{q on the line} w_pq u_q
 *       = F_p + lambda sum_{q off the line} w_pq U_q,
 * F the input, U the estimate the pass starts from (U = F before the first
 * pass); 2 * iters passes in the order of axis_order.  Repeated, it
 * converges to the 2D WLS solution A^-1 F.
 *   f, u  device FP32 C x H x W (u may alias neither f nor g); g: device
 *         FP32 H x W guidance
 *   p     as sgwls_filter; FP32 storage, r <= 4, step 1, no refinement, one
 *         guidance plane (else SGWLS_E_UNSUPPORTED)
 *   ws    workspace of sgwls_line_relax_workspace_bytes bytes, 256-byte
 *         aligned.  Asynchronous on `stream`. */
size_t sgwls_line_relax_workspace_bytes(int H, int W, int C, const sgwls_params* p);
sgwls_status sgwls_line_relax(const void* f, const void* g, void* u, int H, int W, int C, float lambda,
                              const sgwls_params* p, void* ws, size_t ws_bytes, void* stream);

/* One image of a batched backward (all pointers device pointers, FP32). */
typedef struct {
  const float* grad_u;   /* C x H x W, dLoss/du                                  */
  const float* g;        /* H x W guidance of the forward call                   */
  const float* saved;    /* 2*iters*C*H*W checkpoints of the forward call          */
  float* grad_f;         /* C x H x W output, dLoss/df (may not alias grad_u)       */
  float* grad_g;         /* H x W output, dLoss/dg, or NULL                        */
  float* grad_lambda;    /* one float, dLoss/dlambda, or NULL                      */
  int H, W, C;           /* any channel count 1 <= C <= SGWLS_C_MAX                 */
  float lambda;          /* the image's lambda of the forward call                  */
} sgwls_grad_image;

/* Workspace bytes sgwls_filter_backward_batched needs (0 if the arguments
 * are invalid).  Host-only; `imgs` is a host array. */
size_t sgwls_backward_batched_workspace_bytes(int B, const sgwls_grad_image* imgs, const sgwls_params* p);

/* Reverse-mode derivative of a batched forward (sgwls_filter_batched with
 * checkpoints) for B images of uneven sizes and channel counts: per image
 * what sgwls_filter_backward computes (the paper has no backward pass; the
 * chain rule through Eqs. 2, 4, 5 and Sec. 2.3), with every pass of every
 * image run together: one launch that divides each image's dLoss/d(pass
 * output) by its subsystem counts, then one launch per kernel over the
 * channel groups (u and v of up to three channels at r = 1, two otherwise,
 * solved against one factorisation) of all images, per group size.
 * Parameters as sgwls_filter_backward (FP32 storage; frac weights need
 * alpha_r >= 1); ws: sgwls_backward_batched_workspace_bytes bytes, 256-byte
 * aligned.  Gradients w.r.t. g and lambda are accumulated with
 * floating-point atomics: their last bits depend on the order of
 * accumulation. */
sgwls_status sgwls_filter_backward_batched(int B, const sgwls_grad_image* imgs, const sgwls_params* p, void* ws,
                                           size_t ws_bytes, void* stream);

/* One pass like sgwls_filter_pass, for callers that cannot allocate device
 * memory when they filter (a host with a fixed device-memory budget, or a
 * code path that must not enter the allocator): it takes no workspace.  The
 * paper has no counterpart; this is an interface convenience.
 *   Scratch: a file-scope device array of 16 MiB inside libsgwls.so.
 *   Requests whose scratch (sgwls_workspace_bytes with iters = 0 and
 *   factor_cache = 2) exceeds 16 MiB return SGWLS_E_WORKSPACE; e.g. RGB FP32
 *   at r = 1 fits up to about 1920 x 1080.
 *   Set-up: the first call on a device loads the library's device code on
 *   that device, which reserves the 16 MiB there (held until the process
 *   exits), and looks up the array's device address with that device current
 *   (cudaGetSymbolAddress); later calls reuse the address.  Callers under a
 *   memory budget should therefore make one call per device during their own
 *   set-up, and that first call must come before any stream capture.
 *   Sharing: all calls share the one array and leave their contents in it;
 *   each call clears the array's small block-counter region on its stream
 *   before its kernels (every other value the kernels read is written
 *   earlier in the same call); calls that overlap on the GPU (other streams,
 *   other host threads) race on it -- serialise them.
 *   Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *   Checks: the parameters are validated as sgwls_filter_pass validates them
 *   (same codes); then step > 1, refine = 1, guide_channels > 1 and
 *   factor_cache = 1 (kept factors, which the scratch cannot hold) return
 *   SGWLS_E_UNSUPPORTED; u may alias neither f nor g.
 * Other arguments and results as sgwls_filter_pass. */
sgwls_status sgwls_filter_pass_noalloc(const void* f, const void* g, void* u, int H, int W, int C,
                                       float lambda, const sgwls_params* p, int direction, void* stream);

/* Device error flag of the current device.  The queue-scheduled forward
 * pass (schedule = 2 in sgwls_params) runs as one persistent kernel whose
 * blocks wait for
 * one another's work items; every such wait is bounded (at least 2^20 polls
 * and 2 s), and a wait that gives up sets this flag and skips its item, so
 * the kernel always ends but that call's output is not valid.  The flag
 * stays set (later queue-scheduled passes then skip their work at once)
 * until it is cleared.  Every wait is on work that an already running
 * block holds, so a correct run never sets it.
 *   clear  nonzero: clear the flag after reading it
 * Returns SGWLS_OK (flag clear), SGWLS_E_DEVICE_FLAG (flag set) or
 * SGWLS_E_CUDA.  Synchronises with the device (a blocking copy). */
sgwls_status sgwls_device_flag(int clear);

/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all devices).  Diagnostics: lets a caller count the kernels
 * behind a sequence of calls.  Host-only. */
unsigned long long sgwls_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SGWLS_H */
