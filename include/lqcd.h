/*
 * liblqcd -- GB300 (sm_103a) molecular-dynamics hot path of the one-loop
 * Symanzik improved gauge action (D. Li, "The Calculation of Force in Lattice
 * Quantum Chromodynamics", Sec. II), and the hopping operator of the Wilson
 * fermion matrix with its force on the links (Sec. III).
 *
 * C ABI: plain pointers and sizes.  Device buffers are owned by the caller;
 * no entry point allocates device memory, and none synchronises the device
 * except the two that time kernels (lqcd_autotune_force,
 * lqcd_measure_fma_rate); every kernel is enqueued on the caller's stream
 * (`stream` = a cudaStream_t, NULL for the legacy default stream).  Every entry point
 * returns LQCD_OK (0) or a negative LQCD_ERR_* code; arguments are checked
 * before anything is enqueued, so on an argument error no output is touched.
 * LQCD_ERR_CUDA reports a failed launch (the CUDA error is kept for
 * lqcd_last_cuda_error()).
 *
 * Lattice and conventions
 *   Periodic lattice L0 x L1 x L2 x L3 (x, y, z, t), site
 *   n = x + L0*(y + L1*(z + L2*t)), V = L0*L1*L2*L3 sites, 4V links.
 *   U_{n,mu} is the SU(3) link from n to n+mu; U_{n+mu,-mu} = U_{n,mu}^dagger.
 *   T_a = lambda_a/2 (Gell-Mann), a = 0..7 (the paper's i = 1..8),
 *   tr(T_a T_b) = delta_ab/2 (Eq. 18_1_29_3_0).
 *
 * Memory layouts (structure of arrays, `W` = 16 bytes / sizeof(real), i.e.
 * W = 4 for LQCD_F32 (float4 lanes), W = 2 for LQCD_F64 (double2 lanes)):
 *   links  : the first two rows of every link, 12 reals
 *              r = (Re U00, Im U00, Re U01, Im U01, Re U02, Im U02,
 *                   Re U10, Im U10, Re U11, Im U11, Re U12, Im U12),
 *            real r of link (n, mu) at index ((mu*(12/W) + r/W)*V + n)*W + r%W.
 *            The third row is rebuilt as conj(row0 x row1) on every load.
 *            4*12*V reals.
 *   algebra: (force, momenta, omega) 8 reals per link, component a of link
 *            (n, mu) at ((mu*(8/W) + a/W)*V + n)*W + a%W.  4*8*V reals.
 *   full   : (lqcd_pack_links / lqcd_unpack_links only) complex 3x3 links,
 *            [V][4][3][3] of (re, im) pairs, row-major.  4*18*V reals.
 *   All device pointers must be 16-byte aligned (LQCD_ERR_ALIGN otherwise).
 *
 * Force and momenta sign contract (Eqs. 18_7_25_1, 18_7_26_1, 18_7_25_2):
 *   f^a_{n,mu} = -dS_G/domega^a_{n,mu}, the derivative taken along the left
 *   perturbation U -> exp(i eps T_a) U.  As a matrix, the paper's Hermitian
 *   force is sum_a f^a T_a = (beta/6) i (U_{n,mu} t_{n,mu})_TA, with t the
 *   coefficient-weighted sum of the 48 staples of the link.
 *   Molecular dynamics: p^a += dt f^a; U <- exp(i dt sum_a p^a T_a) U.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LQCD_API __attribute__((visibility("default")))
#else
#define LQCD_API
#endif

#define LQCD_VERSION 1

/* Status codes. */
#define LQCD_OK 0
#define LQCD_ERR_ARG (-1)         /* NULL pointer, unknown enum, bad parameter  */
#define LQCD_ERR_DIMS (-2)        /* extent < 1 or 4V*12 reals do not fit int64  */
#define LQCD_ERR_ALIGN (-3)       /* a device pointer is not 16-byte aligned    */
#define LQCD_ERR_WORKSPACE (-4)   /* workspace NULL or smaller than required    */
#define LQCD_ERR_CUDA (-5)        /* a CUDA runtime call or launch failed       */
#define LQCD_ERR_UNSUPPORTED (-6) /* option not available for this precision    */
#define LQCD_ERR_CAPACITY (-7)    /* the launch needs more scratch than the
                                     library's fixed device buffer holds        */

/* Precision of every real in every buffer passed with a descriptor. */
#define LQCD_F32 0
#define LQCD_F64 1

/* Force algorithms (lqcd_desc.force_algo). */
#define LQCD_FORCE_AUTO 0     /* STAPLE_FIELDS when the call gets a large enough
                                 workspace, else FACTORED                       */
#define LQCD_FORCE_PATHS 1    /* one thread per link walks the 48 staples of a
                                 per-direction path table (plain form)          */
#define LQCD_FORCE_FACTORED 2 /* one thread per link, staples regrouped by their
                                 shared end links (134 instead of 180 matrix
                                 products per link)                             */
#define LQCD_FORCE_STAPLE_FIELDS 3 /* two passes: the 24 plaquette staples of
                                 every site are stored in the workspace, then
                                 every staple of a link is built from them (63
                                 products per link); yields the action too     */

/* Problem descriptor.  beta is the inverse coupling of Eq. 18_6_4_1 and
 * (c_plaq, c_rect, c_cube) are the loop coefficients c_P of Eq. 18_3_27_30;
 * lqcd_symanzik_coefficients() fills them from the tadpole factor u0. */
typedef struct lqcd_desc {
    int32_t dims[4];    /* L0..L3, each >= 1                                 */
    int32_t precision;  /* LQCD_F32 or LQCD_F64                              */
    int32_t force_algo; /* LQCD_FORCE_*                                      */
    double beta;
    double c_plaq;
    double c_rect;
    double c_cube;
} lqcd_desc;

/* Loop coefficients of Eq. 18_3_27_30 (host only, no device work):
 *   alpha_s = -4 ln(u0) / 3.06839,  c_plaq = 1,
 *   c_rect = -(1 + 0.4805 alpha_s) / (20 u0^2),
 *   c_cube = -2 * 0.03325 alpha_s / u0^2   (the printed factor 2 is kept).
 * u0 must be finite and > 0.  Any output pointer may be NULL. */
LQCD_API int lqcd_symanzik_coefficients(double u0, double *alpha_s, double *c_plaq, double *c_rect,
                               double *c_cube);

/* Links from their algebra parameters, U_{n,mu} = exp(i sum_a omega^a T_a)
 * (Eq. 18_1_29_3).  omega: algebra layout (device, read); links: link layout
 * (device, written).  The exponential is the Cayley-Hamilton form
 * f0 + f1 Q + f2 Q^2 (exact for 3x3), coefficients by their power series. */
LQCD_API int lqcd_links_from_omega(const lqcd_desc *desc, const void *omega, void *links, void *stream);

/* Gauge force of the Symanzik action for every link (Eq. 18_7_25_2 and the
 * force algorithm of Sec. II): f^a = -dS/domega^a.  links: link layout
 * (device, read); force: algebra layout (device, written).  workspace: device
 * scratch, 256-byte aligned, of lqcd_workspace_bytes(desc) bytes for
 * LQCD_FORCE_STAPLE_FIELDS (LQCD_ERR_WORKSPACE if missing or short); the
 * other algorithms ignore it, and LQCD_FORCE_AUTO uses the staple-field
 * algorithm only when the workspace is large enough. */
LQCD_API int lqcd_gauge_force(const lqcd_desc *desc, const void *links, void *force, void *workspace,
                     size_t workspace_bytes, void *stream);

/* The force, fused with the momentum step: p^a += dt f^a, without storing f.
 * links: link layout (read); mom: algebra layout (read and written).  Uses a
 * workspace-free algorithm (AUTO means FACTORED here). */
LQCD_API int lqcd_gauge_force_update_momenta(const lqcd_desc *desc, const void *links, void *mom,
                                    double dt, void *stream);

/* One force evaluation of an MD step, with optional fused consumers:
 *   force  != NULL: f written (algebra layout, device);
 *   mom    != NULL: p^a += dt f^a (algebra layout, read and written);
 *   action != NULL: S_G of the same links written (one device double, FP64).
 * At least one of the three must be set.  With LQCD_FORCE_STAPLE_FIELDS (or
 * AUTO and a large enough workspace) the action is a by-product of the force
 * pass; otherwise the action kernel of lqcd_gauge_action runs after the force.
 * workspace: lqcd_workspace_bytes(desc) bytes, 256-byte aligned (required
 * for the staple-field algorithm and whenever action != NULL). */
LQCD_API int lqcd_md_force_step(const lqcd_desc *desc, const void *links, void *force, void *mom,
                       double dt, double *action, void *workspace, size_t workspace_bytes,
                       void *stream);

/* Schedules of the force kernels.  An algorithm may come in several
 * variants that compute the same result with a different traversal,
 * storage or register budget (LQCD_FORCE_STAPLE_FIELDS / AUTO: 9; the
 * others: 1).  The choice
 * is process-wide per precision.
 *   lqcd_force_variant_count: number of variants for desc->force_algo.
 *   lqcd_get_force_variant / lqcd_set_force_variant: the current choice;
 *     -1 restores the built-in default, which depends on the precision (and
 *     may depend on the extents in desc: get returns the schedule a launch
 *     with desc would use).  Not thread-safe against concurrent force
 *     launches of the same precision.
 *   lqcd_autotune_force: times every variant `reps` times on these links
 *     (with the fused action, as in an MD step) and keeps the fastest.  It
 *     SYNCHRONISES the stream (call it once at set-up).  force: a scratch
 *     buffer in algebra layout, overwritten; workspace as for the force.
 *     best: the chosen variant; ms: if not NULL, one mean time per variant. */
LQCD_API int lqcd_force_variant_count(const lqcd_desc *desc);
LQCD_API int lqcd_get_force_variant(const lqcd_desc *desc);
LQCD_API int lqcd_set_force_variant(const lqcd_desc *desc, int variant);
LQCD_API int lqcd_autotune_force(const lqcd_desc *desc, const void *links, void *force, void *workspace,
                        size_t workspace_bytes, int reps, void *stream, int *best, float *ms);

/* Batches: up to LQCD_MAX_BATCH lattices of any extents (and the same
 * precision and action parameters, taken from the descriptor; desc->dims is
 * ignored) in ONE persistent launch per pass.  Each entry names its lattice:
 *   dims   extents of this lattice;
 *   links  link layout (force step: read; link step: read and written);
 *   mom    algebra layout (force step: p += dt f if set; link step: read);
 *   force  algebra layout, f written if set (force step);
 *   action one device double, S_G written if set (force step).
 * lqcd_md_force_step_batched uses the staple-field algorithm (force_algo
 * AUTO or STAPLE_FIELDS, else LQCD_ERR_UNSUPPORTED) with a workspace of
 * lqcd_workspace_bytes_batched bytes (the single-lattice workspaces back to
 * back); every lattice gets exactly the result of its own
 * lqcd_md_force_step, bit for bit.  lqcd_md_update_links_batched is the link
 * step U <- exp(i dt p.T) U of every lattice. */
#define LQCD_MAX_BATCH 64
typedef struct lqcd_lattice_ref {
    int32_t dims[4];
    int32_t reserved[4];
    const void *links;
    void *mom;
    void *force;
    double *action;
} lqcd_lattice_ref;

LQCD_API size_t lqcd_workspace_bytes_batched(const lqcd_desc *desc, int n,
                                             const lqcd_lattice_ref *lats);
LQCD_API int lqcd_md_force_step_batched(const lqcd_desc *desc, int n, const lqcd_lattice_ref *lats,
                                        double dt, void *workspace, size_t workspace_bytes,
                                        void *stream);
LQCD_API int lqcd_md_update_links_batched(const lqcd_desc *desc, int n,
                                          const lqcd_lattice_ref *lats, double dt, void *stream);

/* Gauge action S_G = (beta/3) sum_n sum_{34 loops P} c_P [3 - Re tr P_n]
 * (Eq. 18_6_4_1).  links: link layout (device, read).  action: ONE double in
 * device memory (written, FP64 in both precisions: per-loop terms and all
 * sums are accumulated in double, in a fixed order, so the result is
 * bitwise reproducible).  workspace: device scratch of at least
 * lqcd_workspace_bytes(desc) bytes, 256-byte aligned, used for per-block
 * partial sums. */
LQCD_API int lqcd_gauge_action(const lqcd_desc *desc, const void *links, double *action, void *workspace,
                      size_t workspace_bytes, void *stream);

/* Allocation-free form of lqcd_gauge_action, for callers that cannot
 * allocate device memory at all: for example a host application that owns
 * every byte of device memory through its own pool and hands a plug-in only
 * the buffers it computes on, or a loop with a fixed memory budget where an
 * extra cudaMalloc (which may also synchronise the device) is not allowed.
 * The paper has no counterpart; it is an interface convenience.
 *
 * Same result as lqcd_gauge_action (the same kernels and the same number of
 * per-block partial sums, so the value is bitwise identical), but the
 * partial sums go to a scratch array of 4096 doubles (32 KiB) that the
 * library keeps in device memory as a file-scope variable; every device
 * that loads the library holds it until the process exits.  The entry point
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture.
 *   - All calls share the one array.  Every call overwrites the partial sums
 *     it reads, so nothing has to be cleared between calls, but two calls
 *     that overlap on the GPU (different streams, or different host threads
 *     without ordering) race on it and may both return wrong values.
 *   - A device whose reduction grid needs more than 4096 partial sums (more
 *     than 1024 SMs) is rejected with LQCD_ERR_CAPACITY.
 * links: link layout (device, read); action: one double in device memory. */
LQCD_API int lqcd_gauge_action_noalloc(const lqcd_desc *desc, const void *links, double *action,
                              void *stream);

/* Kinetic term K = (1/2) sum_{links, a} p^a p^a of the MD Hamiltonian, in
 * double, same reduction as lqcd_gauge_action.  mom: algebra layout (read);
 * energy: one double in device memory (written). */
LQCD_API int lqcd_kinetic_energy(const lqcd_desc *desc, const void *mom, double *energy, void *workspace,
                        size_t workspace_bytes, void *stream);

/* Momentum step p^a += dt f^a for every link (the equation of motion of
 * H = K + S_G with f = -dS/domega, Eq. 18_7_25_1).  mom: algebra layout (read
 * and written); force: algebra layout (read).  mom == force is rejected. */
LQCD_API int lqcd_md_update_momenta(const lqcd_desc *desc, void *mom, const void *force, double dt,
                           void *stream);

/* Link step U <- exp(i dt sum_a p^a T_a) U for every link (the flow of the
 * left parametrisation of Eq. 18_1_29_3), then Gram-Schmidt of rows 0, 1
 * (row 2 is always rebuilt as conj(row0 x row1)).  links: link layout (read
 * and written); mom: algebra layout (read). */
LQCD_API int lqcd_md_update_links(const lqcd_desc *desc, void *links, const void *mom, double dt,
                         void *stream);

/* Gradient of S with respect to the algebra parameters of the links,
 * for S as a function of omega through U = exp(i omega.T) U0 (Eq. 18_1_29_3):
 *   grad^a = dS/domega^a = components of phi(-ad_X)(-i f.T),  X = i omega.T,
 * phi(z) = (e^z - 1)/z, where f is the force of lqcd_gauge_force evaluated at
 * U (the left derivative of Eqs. 18_7_25_1, 18_7_26_1).  At omega = 0 this is
 * -f.  omega, force: algebra layout (read); grad: algebra layout (written). */
LQCD_API int lqcd_omega_gradient(const lqcd_desc *desc, const void *omega, const void *force, void *grad,
                        void *stream);

/* Precision conversion of a link field (lqcd_convert_links, 12 stored reals
 * per link) or an algebra field (lqcd_convert_algebra, 8 per link) from
 * desc->precision to dst_precision, value by value (FP32 -> FP64 is exact;
 * FP64 -> FP32 rounds to nearest).  Used to evaluate FP32-stored links with
 * FP64 arithmetic (the Metropolis action of an FP32 trajectory).
 * src, dst: device, the two layouts of the two precisions; src != dst. */
LQCD_API int lqcd_convert_links(const lqcd_desc *desc, const void *src, int dst_precision,
                                void *dst, void *stream);
LQCD_API int lqcd_convert_algebra(const lqcd_desc *desc, const void *src, int dst_precision,
                                  void *dst, void *stream);

/* Layout conversions between full complex 3x3 links ([V][4][3][3] (re, im))
 * and the compact link layout, in the descriptor's precision.  pack drops
 * row 2 (the input must be SU(3) for the result to mean the same links);
 * unpack rebuilds it. */
LQCD_API int lqcd_pack_links(const lqcd_desc *desc, const void *full, void *links, void *stream);
LQCD_API int lqcd_unpack_links(const lqcd_desc *desc, const void *links, void *full, void *stream);

/* lqcd_unitarity_deviation: max over links of the departure of the stored
 * links from SU(3), evaluated in FP64 whatever desc->precision is:
 * max(| |r0|^2 - 1 |, | |r1|^2 - 1 |, |<r0, r1>|, | |r2|^2 - 1 |) for the
 * stored rows r0, r1 and the rebuilt r2 = conj(r0 x r1) (|r2|^2 = det U);
 * zero exactly when U^dag U = 1 and det U = 1.  The check of FP32 links
 * across a trajectory.  deviation: device double (8-byte aligned), written;
 * workspace as for lqcd_kinetic_energy.  Deterministic.
 * lqcd_reunitarise_links: Gram-Schmidt of rows 0 and 1 of every link (row 2
 * is always rebuilt) computed in FP64 and rounded to desc->precision, in
 * place.  Neither is in the paper (which fixes no reunitarisation). */
LQCD_API int lqcd_unitarity_deviation(const lqcd_desc *desc, const void *links, double *deviation,
                                      void *workspace, size_t workspace_bytes, void *stream);
LQCD_API int lqcd_reunitarise_links(const lqcd_desc *desc, void *links, void *stream);

/* Gaussian momenta for the momentum refresh of an HMC trajectory: every
 * component p^a_{n,mu} ~ N(0, 1), written in the algebra layout (device,
 * overwritten).  Counter-based, so the field depends only on `seed`:
 * component a of link (n, mu) is standard normal number j = (n*4 + mu)*8 + a
 * of the SplitMix64 stream `seed` (Steele, Lea & Flood 2014: word i =
 * mix(seed + (i+1) * 0x9E3779B97F4A7C15)), by the Box-Muller transform
 * (cosine branch) of words 2j and 2j+1 taken as the 53-bit uniforms
 * u1 = ((w >> 11) + 1) * 2^-53 and u2 = (w >> 11) * 2^-53; computed in FP64
 * and rounded to desc->precision.  Not from the paper (which fixes no HMC
 * driver).  Errors: LQCD_ERR_ARG, LQCD_ERR_ALIGN, LQCD_ERR_DIMS. */
LQCD_API int lqcd_gaussian_momenta(const lqcd_desc *desc, uint64_t seed, void *mom, void *stream);

/* ---------------------------------------------- Wilson fermion (Sec. III)
 *
 * Spinor fields hold 4 (Dirac) x 3 (colour) complex numbers per site:
 * real r = 2*(3*alpha + a) + (0 re, 1 im), r = 0..23, of site n at
 * ((r/W)*V + n)*W + r%W (W = 4 floats or 2 doubles), i.e. 24*V reals in
 * 16-byte lanes like the links; device memory, 16-byte aligned.  The paper
 * fixes no representation of the Euclidean gamma matrices; the library uses
 * the chiral basis (gamma_mu along x, y, z, t = directions 0..3):
 *   gamma_x = [[0,0,0,i],[0,0,i,0],[0,-i,0,0],[-i,0,0,0]]
 *   gamma_y = [[0,0,0,-1],[0,0,1,0],[0,1,0,0],[-1,0,0,0]]
 *   gamma_z = [[0,0,i,0],[0,0,0,-i],[-i,0,0,0],[0,i,0,0]]
 *   gamma_t = [[0,0,1,0],[0,0,0,1],[1,0,0,0],[0,1,0,0]]
 * Only desc->dims and desc->precision are read by these calls.
 *
 * lqcd_wilson_dslash: y = a x + b calD x with the hopping operator of
 * Eq. 18_7_17_4,
 *   (calD x)_n = sum_mu (1 - gamma_mu) U_{n,mu} x_{n+mu}
 *              + (1 + gamma_mu) U_{n-mu,mu}^dagger x_{n-mu}  (periodic).
 * a = 1, b = -kappa gives Y = D X of Eq. 18_7_17_2 without the clover term.
 * x (read) and y (written) must not overlap; a, b finite. */
LQCD_API int lqcd_wilson_dslash(const lqcd_desc *desc, const void *links, const void *x, double a,
                                double b, void *y, void *stream);

/* lqcd_wilson_hopping_force: the hopping-term force of Eqs. 18_1_29_19 to
 * 18_7_17_30 on every link (k, rho):
 *   B = ((1 - gamma_rho) U_{k,rho} X_{k+rho}) (x) Y_k^dagger,
 *   C = X_k (x) (Y_{k+rho}^dagger (1 + gamma_rho) U_{k,rho}^dagger)
 * (outer products in colour, summed over the Dirac index), and the
 * components h^i of the Hermitian matrix -i (B - C)_TA = sum_i T_i h^i,
 * h^i = -(tr(i T_i (B - C)) + c.c.).  The result is f = coef * h: with
 * X = (D^dagger D)^{-1} phi, Y = D X and D = A - kappa calD, coef = kappa
 * gives the hopping part of -d/domega [phi^dagger (D^dagger D)^{-1} phi]
 * (Eq. 18_6_24_0), the term to add to the gauge force.
 * X, Y: spinor layout (read).  force: algebra layout, written if not NULL;
 * mom: algebra layout, mom += dt * f if not NULL (at least one of the two).
 * coef, dt finite.  The outputs must not overlap the inputs. */
LQCD_API int lqcd_wilson_hopping_force(const lqcd_desc *desc, const void *links, const void *X,
                                       const void *Y, double coef, void *force, void *mom,
                                       double dt, void *stream);

/* ------------------------------------------------------------ diagnostics
 *
 * lqcd_measure_fma_rate: the FP32 (precision LQCD_F32) or FP64 (LQCD_F64)
 * FMA issue rate of the current device in TFLOP/s (2 flops per FMA), from a
 * grid that fills every SM with independent FMA chains, timed with CUDA
 * events on `stream` (about 20 ms; synchronises the stream).  The
 * denominators of the ALU-bound force kernels; the paper has no
 * counterpart.  scratch: device, >= lqcd_fma_rate_scratch_bytes() bytes,
 * overwritten.  Returns LQCD_ERR_ARG on a bad precision or NULL output,
 * LQCD_ERR_WORKSPACE if scratch is missing or too small. */
LQCD_API int lqcd_measure_fma_rate(int precision, void *scratch, size_t scratch_bytes,
                                   double *tflops, void *stream);
LQCD_API size_t lqcd_fma_rate_scratch_bytes(void);

/* Bytes of device workspace that this descriptor needs on the current
 * device: the staple planes and action partials of the staple-field force
 * (force_algo STAPLE_FIELDS or AUTO; 24 SU(3) planes per site -- 1728 bytes
 * in FP32, 3456 in FP64, room for either storage form, with V rounded up to
 * a multiple of 32 -- plus one double per 32 sites) and the partial sums of
 * lqcd_gauge_action / lqcd_kinetic_energy (0 on a bad descriptor).  The
 * staple-field algorithm indexes sites with 32-bit integers: for V >= 2^31
 * it returns LQCD_ERR_DIMS (AUTO then takes the factored algorithm). */
LQCD_API size_t lqcd_workspace_bytes(const lqcd_desc *desc);

/* Human-readable text of a status code (static storage). */
LQCD_API const char *lqcd_strerror(int status);

/* The last CUDA error code seen by this library on the calling thread. */
LQCD_API int lqcd_last_cuda_error(void);

/* LQCD_VERSION of the built library. */
LQCD_API int lqcd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LQCD_H */
