// C-ABI entry points of liblqcd (declared in include/lqcd.h): argument
// checks, then one enqueue on the caller's stream.  Nothing here allocates
// device memory or synchronises.
#include <cmath>
#include <cstdint>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

namespace {

// An NVTX range named after the entry point around every C-ABI call (a
// no-op unless a profiler is attached), so that traces group each call's
// kernels under the call that enqueued them.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
};
#define LQCD_TRACE() const TraceRange lqcd_trace_range_(__func__)

thread_local int g_last_cuda_error = 0;

} // namespace

namespace lqcd {

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return LQCD_OK;
    g_last_cuda_error = (int)e;
    return LQCD_ERR_CUDA;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

int check_desc(const lqcd_desc *d)
{
    if (d == nullptr) return LQCD_ERR_ARG;
    if (d->precision != LQCD_F32 && d->precision != LQCD_F64) return LQCD_ERR_ARG;
    if (d->force_algo < LQCD_FORCE_AUTO || d->force_algo > LQCD_FORCE_STAPLE_FIELDS)
        return LQCD_ERR_ARG;
    if (!std::isfinite(d->beta) || !std::isfinite(d->c_plaq) || !std::isfinite(d->c_rect) ||
        !std::isfinite(d->c_cube))
        return LQCD_ERR_ARG;
    // every extent >= 1 and 4 * 18 * V reals addressable with int64 offsets
    const int64_t limit = ((int64_t)1 << 62) / 72;
    int64_t V = 1;
    for (int i = 0; i < 4; ++i) {
        if (d->dims[i] < 1) return LQCD_ERR_DIMS;
        V *= d->dims[i];
        if (V > limit) return LQCD_ERR_DIMS;
    }
    return LQCD_OK;
}

int check_ptrs(std::initializer_list<const void *> ps)
{
    for (const void *p : ps) {
        if (p == nullptr) return LQCD_ERR_ARG;
        if (!aligned16(p)) return LQCD_ERR_ALIGN;
    }
    return LQCD_OK;
}

} // namespace lqcd

namespace {

using lqcd::aligned16;
using lqcd::check_desc;
using lqcd::check_ptrs;
using lqcd::cuda_status;

void copy_dims(int out[4], const lqcd_desc *d)
{
    for (int i = 0; i < 4; ++i) out[i] = d->dims[i];
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

int reduction_setup(const lqcd_desc *desc, void *workspace, size_t workspace_bytes, int *blocks)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    const int b = lqcd::reduction_blocks(dev);
    if (b <= 0) return LQCD_ERR_CUDA;
    if (workspace == nullptr || ((uintptr_t)workspace & 255u) != 0) return LQCD_ERR_WORKSPACE;
    if (workspace_bytes < (size_t)b * sizeof(double)) return LQCD_ERR_WORKSPACE;
    *blocks = b;
    (void)desc;
    return LQCD_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Workspace of the staple-field force: staple planes, then action partials.
size_t staple_workspace_bytes(const lqcd_desc *d)
{
    return lqcd::staple_field_bytes(d->dims, d->precision) +
           round256((size_t)lqcd::staple_force_partials(d->dims) * sizeof(double));
}

bool workspace_fits(const void *ws, size_t have, size_t need)
{
    return ws != nullptr && ((uintptr_t)ws & 255u) == 0 && have >= need;
}

// The force (and its fused consumers) with the algorithm the descriptor and
// the workspace select.  Arguments are already checked.
int run_force(const lqcd_desc *desc, const void *links, void *force, void *mom, double dt,
              double *action, void *workspace, size_t workspace_bytes, void *stream)
{
    int algo = desc->force_algo;
    const bool sf_dims = lqcd::staple_fields_supported(desc->dims);
    if (algo == LQCD_FORCE_STAPLE_FIELDS && !sf_dims) return LQCD_ERR_DIMS;
    const bool sf_ok = sf_dims && workspace_fits(workspace, workspace_bytes, staple_workspace_bytes(desc));
    if (algo == LQCD_FORCE_STAPLE_FIELDS && !sf_ok) return LQCD_ERR_WORKSPACE;
    if (algo == LQCD_FORCE_AUTO) algo = sf_ok ? LQCD_FORCE_STAPLE_FIELDS : LQCD_FORCE_FACTORED;
    int red_blocks = 0;
    if (action != nullptr && algo != LQCD_FORCE_STAPLE_FIELDS) {
        const int s = reduction_setup(desc, workspace, workspace_bytes, &red_blocks);
        if (s) return s;
    }
    lqcd::ForceArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.algo = algo;
    a.beta = desc->beta;
    a.c_plaq = desc->c_plaq;
    a.c_rect = desc->c_rect;
    a.c_cube = desc->c_cube;
    a.links = links;
    a.force = force;
    a.mom = mom;
    a.dt = dt;
    a.variant = -1;
    if (algo == LQCD_FORCE_STAPLE_FIELDS) {
        char *ws = static_cast<char *>(workspace);
        a.staples = ws;
        a.partials = reinterpret_cast<double *>(ws + lqcd::staple_field_bytes(desc->dims, desc->precision));
        a.action = action;
        return cuda_status(lqcd::launch_force_staple_fields(a, as_stream(stream)));
    }
    int s = cuda_status(lqcd::launch_force(a, as_stream(stream)));
    if (s || action == nullptr) return s;
    lqcd::ReduceArgs r{};
    copy_dims(r.dims, desc);
    r.precision = desc->precision;
    r.links = links;
    r.c[0] = desc->c_plaq;
    r.c[1] = desc->c_rect;
    r.c[2] = desc->c_cube;
    r.scale = desc->beta / 3.0;
    r.partials = static_cast<double *>(workspace);
    r.blocks = red_blocks;
    r.out = action;
    return cuda_status(lqcd::launch_action(r, as_stream(stream)));
}

} // namespace

extern "C" {

int lqcd_symanzik_coefficients(double u0, double *alpha_s, double *c_plaq, double *c_rect,
                               double *c_cube)
{
    LQCD_TRACE();
    if (!std::isfinite(u0) || !(u0 > 0.0)) return LQCD_ERR_ARG;
    const double as = -4.0 * std::log(u0) / 3.06839;
    if (alpha_s) *alpha_s = as;
    if (c_plaq) *c_plaq = 1.0;
    if (c_rect) *c_rect = -(1.0 + 0.4805 * as) / (20.0 * u0 * u0);
    if (c_cube) *c_cube = -2.0 * 0.03325 * as / (u0 * u0);
    return LQCD_OK;
}

int lqcd_links_from_omega(const lqcd_desc *desc, const void *omega, void *links, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({omega, links}))) return s;
    if (omega == links) return LQCD_ERR_ARG;
    lqcd::MdArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.links = links;
    a.mom = omega;
    return cuda_status(lqcd::launch_links_from_omega(a, as_stream(stream)));
}

int lqcd_gauge_force(const lqcd_desc *desc, const void *links, void *force, void *workspace,
                     size_t workspace_bytes, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links, force}))) return s;
    if (links == force) return LQCD_ERR_ARG;
    return run_force(desc, links, force, nullptr, 0.0, nullptr, workspace, workspace_bytes, stream);
}

int lqcd_gauge_force_update_momenta(const lqcd_desc *desc, const void *links, void *mom,
                                    double dt, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links, mom}))) return s;
    if (links == mom || !std::isfinite(dt)) return LQCD_ERR_ARG;
    if (desc->force_algo == LQCD_FORCE_STAPLE_FIELDS) return LQCD_ERR_WORKSPACE;
    return run_force(desc, links, nullptr, mom, dt, nullptr, nullptr, 0, stream);
}

int lqcd_md_force_step(const lqcd_desc *desc, const void *links, void *force, void *mom,
                       double dt, double *action, void *workspace, size_t workspace_bytes,
                       void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links}))) return s;
    if (force == nullptr && mom == nullptr && action == nullptr) return LQCD_ERR_ARG;
    if (force != nullptr && ((s = check_ptrs({force})))) return s;
    if (mom != nullptr && ((s = check_ptrs({mom})))) return s;
    if (action != nullptr && ((uintptr_t)action & 7u) != 0) return LQCD_ERR_ALIGN;
    if (links == force || links == mom || (force != nullptr && force == mom)) return LQCD_ERR_ARG;
    if (mom != nullptr && !std::isfinite(dt)) return LQCD_ERR_ARG;
    return run_force(desc, links, force, mom, dt, action, workspace, workspace_bytes, stream);
}

namespace {

// Batched calls: the descriptor supplies precision, coefficients and the
// algorithm; every entry its own extents.
int check_batch(const lqcd_desc *desc, int n, const lqcd_lattice_ref *lats)
{
    int s = check_desc(desc);
    if (s) return s;
    if (n < 1 || n > LQCD_MAX_BATCH || lats == nullptr) return LQCD_ERR_ARG;
    for (int c = 0; c < n; ++c) {
        lqcd_desc d = *desc;
        for (int i = 0; i < 4; ++i) d.dims[i] = lats[c].dims[i];
        if ((s = check_desc(&d))) return s;
        if ((s = check_ptrs({lats[c].links}))) return s;
        if (lats[c].mom != nullptr && !aligned16(lats[c].mom)) return LQCD_ERR_ALIGN;
        if (lats[c].force != nullptr && !aligned16(lats[c].force)) return LQCD_ERR_ALIGN;
        if (lats[c].action != nullptr && ((uintptr_t)lats[c].action & 7u) != 0) return LQCD_ERR_ALIGN;
    }
    return LQCD_OK;
}

size_t batch_workspace_bytes(const lqcd_desc *desc, int n, const lqcd_lattice_ref *lats)
{
    size_t total = 0;
    for (int c = 0; c < n; ++c) {
        lqcd_desc d = *desc;
        for (int i = 0; i < 4; ++i) d.dims[i] = lats[c].dims[i];
        total += staple_workspace_bytes(&d);
    }
    return total + lqcd::kBatchCounterBytes;
}

} // namespace

size_t lqcd_workspace_bytes_batched(const lqcd_desc *desc, int n, const lqcd_lattice_ref *lats)
{
    LQCD_TRACE();
    if (check_batch(desc, n, lats) != LQCD_OK) return 0;
    return batch_workspace_bytes(desc, n, lats);
}

int lqcd_md_force_step_batched(const lqcd_desc *desc, int n, const lqcd_lattice_ref *lats,
                               double dt, void *workspace, size_t workspace_bytes, void *stream)
{
    LQCD_TRACE();
    int s = check_batch(desc, n, lats);
    if (s) return s;
    if (desc->force_algo != LQCD_FORCE_AUTO && desc->force_algo != LQCD_FORCE_STAPLE_FIELDS)
        return LQCD_ERR_UNSUPPORTED;
    if (!std::isfinite(dt)) return LQCD_ERR_ARG;
    for (int c = 0; c < n; ++c) {
        if (lats[c].force == nullptr && lats[c].mom == nullptr && lats[c].action == nullptr)
            return LQCD_ERR_ARG;
        if (!lqcd::staple_fields_supported(lats[c].dims)) return LQCD_ERR_DIMS;
    }
    if (!workspace_fits(workspace, workspace_bytes, batch_workspace_bytes(desc, n, lats)))
        return LQCD_ERR_WORKSPACE;
    lqcd::SfLattice items[LQCD_MAX_BATCH];
    char *ws = static_cast<char *>(workspace);
    for (int c = 0; c < n; ++c) {
        lqcd::SfLattice &L = items[c];
        L = lqcd::SfLattice{};
        for (int i = 0; i < 4; ++i) L.dims[i] = lats[c].dims[i];
        L.links = lats[c].links;
        L.force = lats[c].force;
        L.mom = lats[c].mom;
        L.action = lats[c].action;
        const size_t sf = lqcd::staple_field_bytes(L.dims, desc->precision);
        L.staples = ws;
        L.partials = reinterpret_cast<double *>(ws + sf);
        lqcd_desc d = *desc;
        for (int i = 0; i < 4; ++i) d.dims[i] = lats[c].dims[i];
        ws += staple_workspace_bytes(&d);
    }
    lqcd::ForceArgs a{};
    a.precision = desc->precision;
    a.beta = desc->beta;
    a.c_plaq = desc->c_plaq;
    a.c_rect = desc->c_rect;
    a.c_cube = desc->c_cube;
    a.dt = dt;
    a.variant = -1;
    auto *counter = reinterpret_cast<unsigned long long *>(ws); // after the last lattice's part
    return cuda_status(
        lqcd::launch_force_staple_fields_batched(a, n, items, counter, as_stream(stream)));
}

int lqcd_md_update_links_batched(const lqcd_desc *desc, int n, const lqcd_lattice_ref *lats,
                                 double dt, void *stream)
{
    LQCD_TRACE();
    int s = check_batch(desc, n, lats);
    if (s) return s;
    if (!std::isfinite(dt)) return LQCD_ERR_ARG;
    lqcd::LinkStepItem items[LQCD_MAX_BATCH];
    for (int c = 0; c < n; ++c) {
        if (lats[c].mom == nullptr || lats[c].mom == lats[c].links) return LQCD_ERR_ARG;
        items[c].V = (int64_t)lats[c].dims[0] * lats[c].dims[1] * lats[c].dims[2] * lats[c].dims[3];
        items[c].links = const_cast<void *>(lats[c].links);
        items[c].mom = lats[c].mom;
    }
    return cuda_status(
        lqcd::launch_update_links_batched(desc->precision, n, items, dt, as_stream(stream)));
}

int lqcd_force_variant_count(const lqcd_desc *desc)
{
    LQCD_TRACE();
    const int s = check_desc(desc);
    if (s) return s;
    const bool sf = desc->force_algo == LQCD_FORCE_AUTO || desc->force_algo == LQCD_FORCE_STAPLE_FIELDS;
    return sf ? lqcd::staple_force_variants() : 1;
}

int lqcd_get_force_variant(const lqcd_desc *desc)
{
    LQCD_TRACE();
    const int s = check_desc(desc);
    if (s) return s;
    const bool sf = desc->force_algo == LQCD_FORCE_AUTO || desc->force_algo == LQCD_FORCE_STAPLE_FIELDS;
    return sf ? lqcd::staple_force_variant(desc->precision, desc->dims) : 0;
}

int lqcd_set_force_variant(const lqcd_desc *desc, int variant)
{
    LQCD_TRACE();
    const int s = check_desc(desc);
    if (s) return s;
    const bool sf = desc->force_algo == LQCD_FORCE_AUTO || desc->force_algo == LQCD_FORCE_STAPLE_FIELDS;
    const int count = sf ? lqcd::staple_force_variants() : 1;
    if (variant < -1 || variant >= count) return LQCD_ERR_ARG;
    if (sf) lqcd::set_staple_force_variant(desc->precision, variant);
    return LQCD_OK;
}

int lqcd_autotune_force(const lqcd_desc *desc, const void *links, void *force, void *workspace,
                        size_t workspace_bytes, int reps, void *stream, int *best, float *ms)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links, force}))) return s;
    if (links == force || reps < 1) return LQCD_ERR_ARG;
    const bool sf = desc->force_algo == LQCD_FORCE_AUTO || desc->force_algo == LQCD_FORCE_STAPLE_FIELDS;
    if (!sf) {
        if (best) *best = 0;
        return LQCD_OK;
    }
    if (!lqcd::staple_fields_supported(desc->dims)) return LQCD_ERR_DIMS;
    if (!workspace_fits(workspace, workspace_bytes, staple_workspace_bytes(desc)))
        return LQCD_ERR_WORKSPACE;
    lqcd_desc d = *desc;
    d.force_algo = LQCD_FORCE_STAPLE_FIELDS;
    double *action = static_cast<double *>(force); // scratch: force[0] receives the action
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    const int count = lqcd::staple_force_variants();
    int arg = 0;
    float best_ms = 0.f;
    for (int v = 0; v < count && ce == cudaSuccess && s == LQCD_OK; ++v) {
        lqcd::set_staple_force_variant(desc->precision, v);
        s = run_force(&d, links, force, nullptr, 0.0, action, workspace, workspace_bytes, stream);
        if (s) break;
        float acc = 0.f;
        for (int r = 0; r < reps && s == LQCD_OK && ce == cudaSuccess; ++r) {
            ce = cudaEventRecord(e0, as_stream(stream));
            if (ce != cudaSuccess) break;
            s = run_force(&d, links, force, nullptr, 0.0, action, workspace, workspace_bytes, stream);
            if (s) break;
            ce = cudaEventRecord(e1, as_stream(stream));
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float t = 0.f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
            acc += t;
        }
        const float mean = acc / (float)reps;
        if (ms) ms[v] = mean;
        if (v == 0 || mean < best_ms) {
            best_ms = mean;
            arg = v;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s == LQCD_OK && ce != cudaSuccess) s = cuda_status(ce);
    lqcd::set_staple_force_variant(desc->precision, s == LQCD_OK ? arg : -1);
    if (best) *best = s == LQCD_OK ? arg : -1;
    return s;
}

int lqcd_gauge_action(const lqcd_desc *desc, const void *links, double *action, void *workspace,
                      size_t workspace_bytes, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links}))) return s;
    if (action == nullptr) return LQCD_ERR_ARG;
    if (((uintptr_t)action & 7u) != 0) return LQCD_ERR_ALIGN;
    int blocks = 0;
    if ((s = reduction_setup(desc, workspace, workspace_bytes, &blocks))) return s;
    lqcd::ReduceArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.links = links;
    a.c[0] = desc->c_plaq;
    a.c[1] = desc->c_rect;
    a.c[2] = desc->c_cube;
    a.scale = desc->beta / 3.0;
    a.partials = static_cast<double *>(workspace);
    a.blocks = blocks;
    a.out = action;
    return cuda_status(lqcd::launch_action(a, as_stream(stream)));
}

int lqcd_kinetic_energy(const lqcd_desc *desc, const void *mom, double *energy, void *workspace,
                        size_t workspace_bytes, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({mom}))) return s;
    if (energy == nullptr) return LQCD_ERR_ARG;
    if (((uintptr_t)energy & 7u) != 0) return LQCD_ERR_ALIGN;
    int blocks = 0;
    if ((s = reduction_setup(desc, workspace, workspace_bytes, &blocks))) return s;
    lqcd::ReduceArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.mom = mom;
    a.partials = static_cast<double *>(workspace);
    a.blocks = blocks;
    a.out = energy;
    return cuda_status(lqcd::launch_kinetic(a, as_stream(stream)));
}

int lqcd_unitarity_deviation(const lqcd_desc *desc, const void *links, double *deviation,
                             void *workspace, size_t workspace_bytes, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links}))) return s;
    if (deviation == nullptr) return LQCD_ERR_ARG;
    if (((uintptr_t)deviation & 7u) != 0) return LQCD_ERR_ALIGN;
    int blocks = 0;
    if ((s = reduction_setup(desc, workspace, workspace_bytes, &blocks))) return s;
    lqcd::ReduceArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.links = links;
    a.partials = static_cast<double *>(workspace);
    a.blocks = blocks;
    a.out = deviation;
    return cuda_status(lqcd::launch_unitarity(a, as_stream(stream)));
}

int lqcd_reunitarise_links(const lqcd_desc *desc, void *links, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links}))) return s;
    lqcd::MdArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.links = links;
    return cuda_status(lqcd::launch_reunitarise(a, as_stream(stream)));
}

int lqcd_md_update_momenta(const lqcd_desc *desc, void *mom, const void *force, double dt,
                           void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({mom, force}))) return s;
    if (mom == force || !std::isfinite(dt)) return LQCD_ERR_ARG;
    lqcd::MdArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.mom_out = mom;
    a.force = force;
    a.dt = dt;
    return cuda_status(lqcd::launch_update_momenta(a, as_stream(stream)));
}

int lqcd_md_update_links(const lqcd_desc *desc, void *links, const void *mom, double dt,
                         void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links, mom}))) return s;
    if (links == mom || !std::isfinite(dt)) return LQCD_ERR_ARG;
    lqcd::MdArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.links = links;
    a.mom = mom;
    a.dt = dt;
    return cuda_status(lqcd::launch_update_links(a, as_stream(stream)));
}

int lqcd_omega_gradient(const lqcd_desc *desc, const void *omega, const void *force, void *grad,
                        void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({omega, force, grad}))) return s;
    if (grad == omega || grad == force) return LQCD_ERR_ARG;
    lqcd::MdArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.mom = omega;
    a.force = force;
    a.mom_out = grad;
    return cuda_status(lqcd::launch_omega_gradient(a, as_stream(stream)));
}

int lqcd_gaussian_momenta(const lqcd_desc *desc, uint64_t seed, void *mom, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({mom}))) return s;
    lqcd::MdArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.mom_out = mom;
    a.seed = seed;
    return cuda_status(lqcd::launch_gaussian_momenta(a, as_stream(stream)));
}

int lqcd_wilson_dslash(const lqcd_desc *desc, const void *links, const void *x, double a, double b,
                       void *y, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links, x, y}))) return s;
    if (x == y || y == links || !std::isfinite(a) || !std::isfinite(b)) return LQCD_ERR_ARG;
    lqcd::WilsonArgs w{};
    copy_dims(w.dims, desc);
    w.precision = desc->precision;
    w.links = links;
    w.x = x;
    w.out = y;
    w.ca = a;
    w.cb = b;
    return cuda_status(lqcd::launch_wilson_dslash(w, as_stream(stream)));
}

int lqcd_wilson_hopping_force(const lqcd_desc *desc, const void *links, const void *X, const void *Y,
                              double coef, void *force, void *mom, double dt, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({links, X, Y}))) return s;
    if (force == nullptr && mom == nullptr) return LQCD_ERR_ARG;
    if (force != nullptr && (s = check_ptrs({force}))) return s;
    if (mom != nullptr && (s = check_ptrs({mom}))) return s;
    if (force != nullptr && force == mom) return LQCD_ERR_ARG;
    for (const void *o : {(const void *)force, (const void *)mom})
        if (o != nullptr && (o == links || o == X || o == Y)) return LQCD_ERR_ARG;
    if (!std::isfinite(coef) || !std::isfinite(dt)) return LQCD_ERR_ARG;
    lqcd::WilsonArgs w{};
    copy_dims(w.dims, desc);
    w.precision = desc->precision;
    w.links = links;
    w.x = X;
    w.y = Y;
    w.force = force;
    w.mom = mom;
    w.coef = coef;
    w.dt = dt;
    return cuda_status(lqcd::launch_wilson_hopping_force(w, as_stream(stream)));
}

int lqcd_measure_fma_rate(int precision, void *scratch, size_t scratch_bytes, double *tflops,
                          void *stream)
{
    LQCD_TRACE();
    if ((precision != LQCD_F32 && precision != LQCD_F64) || tflops == nullptr) return LQCD_ERR_ARG;
    if (scratch == nullptr || scratch_bytes < lqcd::fma_rate_scratch_bytes() || !aligned16(scratch))
        return LQCD_ERR_WORKSPACE;
    return cuda_status(lqcd::measure_fma_rate(precision, scratch, scratch_bytes, tflops,
                                              as_stream(stream)));
}

size_t lqcd_fma_rate_scratch_bytes(void) { return lqcd::fma_rate_scratch_bytes(); }

static int convert_common(const lqcd_desc *desc, const void *src, int dst_precision, void *dst,
                          bool links, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({src, dst}))) return s;
    if (dst_precision != LQCD_F32 && dst_precision != LQCD_F64) return LQCD_ERR_ARG;
    if (src == dst) return LQCD_ERR_ARG;
    lqcd::MdArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.full_in = src;
    a.full_out = dst;
    return cuda_status(lqcd::launch_convert(a, dst_precision, links, as_stream(stream)));
}

int lqcd_convert_links(const lqcd_desc *desc, const void *src, int dst_precision, void *dst,
                       void *stream)
{
    LQCD_TRACE();
    return convert_common(desc, src, dst_precision, dst, true, stream);
}

int lqcd_convert_algebra(const lqcd_desc *desc, const void *src, int dst_precision, void *dst,
                         void *stream)
{
    LQCD_TRACE();
    return convert_common(desc, src, dst_precision, dst, false, stream);
}

int lqcd_pack_links(const lqcd_desc *desc, const void *full, void *links, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({full, links}))) return s;
    if (full == links) return LQCD_ERR_ARG;
    lqcd::MdArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.full_in = full;
    a.links = links;
    return cuda_status(lqcd::launch_pack(a, as_stream(stream)));
}

int lqcd_unpack_links(const lqcd_desc *desc, const void *links, void *full, void *stream)
{
    LQCD_TRACE();
    int s = check_desc(desc);
    if (s) return s;
    if ((s = check_ptrs({full, links}))) return s;
    if (full == links) return LQCD_ERR_ARG;
    lqcd::MdArgs a{};
    copy_dims(a.dims, desc);
    a.precision = desc->precision;
    a.links = const_cast<void *>(links);
    a.full_out = full;
    return cuda_status(lqcd::launch_unpack(a, as_stream(stream)));
}

size_t lqcd_workspace_bytes(const lqcd_desc *desc)
{
    LQCD_TRACE();
    if (check_desc(desc) != LQCD_OK) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const int b = lqcd::reduction_blocks(dev);
    if (b <= 0) return 0;
    size_t need = round256((size_t)b * sizeof(double));
    if (desc->force_algo == LQCD_FORCE_AUTO || desc->force_algo == LQCD_FORCE_STAPLE_FIELDS) {
        const size_t sf = staple_workspace_bytes(desc);
        if (sf > need) need = sf;
    }
    return need;
}

const char *lqcd_strerror(int status)
{
    switch (status) {
    case LQCD_OK: return "success";
    case LQCD_ERR_ARG: return "invalid argument";
    case LQCD_ERR_DIMS: return "invalid lattice extents";
    case LQCD_ERR_ALIGN: return "device pointer not 16-byte aligned";
    case LQCD_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case LQCD_ERR_CUDA: return "CUDA runtime error";
    case LQCD_ERR_UNSUPPORTED: return "unsupported option";
    case LQCD_ERR_CAPACITY: return "problem needs more scratch than the fixed library buffer holds";
    default: return "unknown status";
    }
}

int lqcd_last_cuda_error(void) { return g_last_cuda_error; }

int lqcd_version(void) { return LQCD_VERSION; }

} // extern "C"
