// Internal launch interface between the C-ABI layer (api.cu) and the kernel
// translation units.  Host-side C++ only; no torch types.
#pragma once

#include <cstddef>
#include <cstdint>
#include <initializer_list>
#include <cuda_runtime.h>

#include "../../include/lqcd.h"

namespace lqcd {

// Argument checks shared by every entry point (api.cu): the descriptor
// (precision, algorithm, finite parameters, extents >= 1 and addressable),
// and device pointers (non-NULL: else LQCD_ERR_ARG; 16-byte aligned: else
// LQCD_ERR_ALIGN).  cuda_status maps a CUDA error to LQCD_ERR_CUDA and keeps
// it for lqcd_last_cuda_error() on the calling thread.
int check_desc(const lqcd_desc *d);
int check_ptrs(std::initializer_list<const void *> ps);
bool aligned16(const void *p);
int cuda_status(cudaError_t e);

// One staple of the path kernel: cls (0 plaquette, 1 rectangle, 2 cube),
// len (3 or 5) signed directions +-(mu+1), walked from k + rho.
struct Staple {
    int8_t cls;
    int8_t len;
    int8_t d[6];
};

struct StapleTable {
    Staple s[4][48];
    int count;
};

const StapleTable &staple_table();

// Per-launch scalars computed once on the host, in both precisions, so that
// no kernel thread spends FP64 instructions on them: beta/6, c_plaq, c_rect,
// c_cube, the per-link action constant 3 (1.5 c_plaq + 3 c_rect + 4 c_cube),
// c_plaq/12 and dt.
struct KernelScalars {
    double d[7];
    float f[7];
};

struct ForceArgs {
    int dims[4];
    int precision;
    int algo;
    double beta, c_plaq, c_rect, c_cube;
    const void *links;
    void *force; // written when mom == nullptr
    void *mom;   // when set: mom += dt * f
    double dt;
    void *staples;     // staple-field algorithm: workspace for the 24 staple planes
    double *partials;  // staple-field algorithm with action: per-block partial sums
    double *action;    // staple-field algorithm: action written here when set
    int variant;       // staple-field force pass schedule; -1 = process-wide choice
};

// Unsigned division of n < 2^31 by an invariant d >= 1 (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994):
// t = mulhi(m, n), n / d = (t + ((n - t) >> sh1)) >> sh2 with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, sh1 = min(l, 1), sh2 = max(l - 1, 0);
// the quotient is div_by (su3.cuh).  Kernels take these for the run-time
// extents they divide site indices by, instead of dividing.
struct DivMagic {
    unsigned m;
    int sh1, sh2;
};

inline DivMagic div_magic(unsigned d)
{
    int l = 0;
    while (l < 32 && ((uint64_t)1 << l) < d) ++l;
    DivMagic g;
    g.m = (unsigned)((((uint64_t)1 << 32) * (((uint64_t)1 << l) - d)) / d + 1);
    g.sh1 = l < 1 ? l : 1;
    g.sh2 = l > 1 ? l - 1 : 0;
    return g;
}

// One lattice as the staple-field kernels see it (filled on the host).
struct SfLattice {
    int dims[4];
    int sweep[3];      // spatial block extents of the pass-B traversal
    int micro[3];      // micro-tile extents inside a block slice
    // division magic (set_traversal): site strides L0, L0 L1, L0 L1 L2, then
    // the sweep's block volume, slice, micro-tile volume, micro-tile x and y
    // extents, micro-tiles along x and y of a block, blocks along x and y
    DivMagic div[12];
    int counts[4];     // blocks along x and y, micro-tiles along x and y of a block
    int64_t vb_begin;  // batch: first virtual block of this lattice
    int64_t plane_bytes; // full staple planes: bytes of one plane
    const void *links;
    void *staples;     // 24 staple planes (workspace)
    void *force;       // written when set
    void *mom;         // p += dt f when set
    double *partials;  // one action partial per virtual block
    double *action;    // action written here when set
};

constexpr int kMaxBatch = 64;

struct SfBatch {
    int n;
    int64_t total;                 // virtual blocks of all lattices
    unsigned long long *counter;   // work counters (2, zeroed before the passes)
    SfLattice e[kMaxBatch];
};

// Bytes at the end of a batch workspace for the persistent launches' work
// counters.
constexpr size_t kBatchCounterBytes = 256;

cudaError_t launch_force(const ForceArgs &a, cudaStream_t st);

// Staple-field algorithm (force_sf.cu): workspace bytes of the 24 staple
// planes, number of per-block action partials, and the two-pass launch.
size_t staple_field_bytes(const int dims[4], int precision);
// The staple-field kernels index sites with 32-bit integers: V < 2^31.
bool staple_fields_supported(const int dims[4]);
int staple_force_partials(const int dims[4]);
cudaError_t launch_force_staple_fields(const ForceArgs &a, cudaStream_t st);
// a: precision, coefficients, dt, variant; items: the lattices (their dims,
// links, staples, force, mom, partials, action), 1 <= n <= kMaxBatch.
cudaError_t launch_force_staple_fields_batched(const ForceArgs &a, int n, const SfLattice *items,
                                               unsigned long long *counter, cudaStream_t st);
int staple_force_variants();
int staple_force_variant(int precision, const int dims[4]); // current choice (default by shape)
void set_staple_force_variant(int precision, int variant);

// The 34 loops of the action kernel: cls, len (4 or 6), signed directions.
struct Loop {
    int8_t cls;
    int8_t len;
    int8_t d[6];
};

struct LoopTable {
    Loop l[34];
    int count;
};

const LoopTable &loop_table();

struct ReduceArgs {
    int dims[4];
    int precision;
    const void *links; // action
    const void *mom;   // kinetic energy
    double c[3];
    double scale;      // result = scale * sum
    double *partials;  // workspace, one double per block
    int blocks;
    double *out;
};

int reduction_blocks(int device);
// out = scale * (sum of partials[0..count)), one block, fixed order.
cudaError_t launch_finish_sum(const double *partials, int count, double scale, double *out,
                              cudaStream_t st);
cudaError_t launch_action(const ReduceArgs &a, cudaStream_t st);
cudaError_t launch_kinetic(const ReduceArgs &a, cudaStream_t st);
// out = max over links of the FP64 departure of the stored links from SU(3).
cudaError_t launch_unitarity(const ReduceArgs &a, cudaStream_t st);

struct MdArgs {
    int dims[4];
    int precision;
    void *links;
    const void *mom;
    const void *force;
    void *mom_out;
    const void *full_in;
    void *full_out;
    double dt;
    uint64_t seed; // gaussian momenta: the generator stream
};

cudaError_t launch_update_momenta(const MdArgs &a, cudaStream_t st);
// U <- exp(i dt p.T) U for n lattices in one persistent launch.
struct LinkStepItem {
    int64_t V;
    void *links;
    const void *mom;
};
cudaError_t launch_update_links_batched(int precision, int n, const LinkStepItem *items, double dt,
                                        cudaStream_t st);
cudaError_t launch_update_links(const MdArgs &a, cudaStream_t st);
cudaError_t launch_links_from_omega(const MdArgs &a, cudaStream_t st);
cudaError_t launch_omega_gradient(const MdArgs &a, cudaStream_t st);
// full_in -> full_out in another precision; links: 12 reals per item, else 8
cudaError_t launch_convert(const MdArgs &a, int dst_precision, bool links, cudaStream_t st);
cudaError_t launch_pack(const MdArgs &a, cudaStream_t st);
cudaError_t launch_unpack(const MdArgs &a, cudaStream_t st);
// links <- Gram-Schmidt of rows 0 and 1 in FP64, rounded to the storage precision.
cudaError_t launch_reunitarise(const MdArgs &a, cudaStream_t st);
// mom_out <- Gaussian momenta of stream a.seed (SplitMix64 + Box-Muller).
cudaError_t launch_gaussian_momenta(const MdArgs &a, cudaStream_t st);

// Wilson fermion hopping term (Sec. III).  Spinor fields: 24 reals per site,
// real r = 2*(3*alpha + a) + (0 re, 1 im) of site n at ((r/W)*V + n)*W + r%W.

struct WilsonArgs {
    int dims[4];
    int precision;
    const void *links;
    const void *x;   // dslash input; force: X
    const void *y;   // force: Y
    void *out;       // dslash output
    void *force;     // force output (or null)
    void *mom;       // momenta updated in place (or null)
    double ca, cb;   // dslash: out = ca * x + cb * calD x
    double coef, dt; // force: f = coef * h;  mom += dt * f
    // the same four scalars rounded to FP32 by the launcher, so that FP32
    // kernels spend no FP64 conversions on them
    float fca, fcb, fcoef, fdt;
    // division of a site index (below 2^31) by the strides L0, L0 L1,
    // L0 L1 L2 as a multiply-high and shifts (set by the launcher)
    DivMagic div[3];
};
cudaError_t launch_wilson_dslash(const WilsonArgs &a, cudaStream_t st);
// FMA issue rate of the device in TFLOP/s (synchronises); scratch >= fma_rate_scratch_bytes().
cudaError_t measure_fma_rate(int precision, void *scratch, size_t scratch_bytes, double *tflops,
                             cudaStream_t st);
size_t fma_rate_scratch_bytes();
cudaError_t launch_wilson_hopping_force(const WilsonArgs &a, cudaStream_t st);

} // namespace lqcd
