// Host side of the C ABI declared in include/dgx.h: handle life cycle,
// device buffers, the Runge-Kutta stage schedule, small reduction kernels and
// CUDA-graph replay of whole steps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dgx.h"
#include "dgx_internal.h"

using namespace dgx;

namespace {

// ------------------------------------------------------------------ SSP Runge-Kutta schedules (Sec. 2.5)
//
// Each stage evaluates L at u^n + delta_in and forms, in "delta form",
//   delta_out = ca delta_in + cx X + cb dt L,   X <- za delta_in + zx X + zb dt L (optional),
// where X is an auxiliary register; the last stage commits u^{n+1} = u^n + delta_out in FP64.
// The delta form is the Shu-Osher form rewritten with u_i = u^n + delta_i, using that the
// coefficients of each Shu-Osher row sum to one.
struct StageDesc {
    double ca, cx, cb, za, zx, zb;
    int in, out, x, write_z, last;
};

struct Schedule {
    int stages;
    StageDesc s[5];
};

Schedule schedule_for(int stages)
{
    Schedule S{};
    S.stages = stages;
    switch (stages) {
    case 1:  // forward Euler
        S.s[0] = {0, 0, 1, 0, 0, 0, -1, -1, -1, 0, 1};
        break;
    case 2:  // SSP-RK2 (Heun): u1 = u + dt L(u); u2 = u/2 + u1/2 + dt L(u1)/2
        S.s[0] = {0, 0, 1, 0, 0, 0, -1, 0, -1, 0, 0};
        S.s[1] = {0.5, 0, 0.5, 0, 0, 0, 0, -1, -1, 0, 1};
        break;
    case 3:  // SSP-RK3 (Shu-Osher): u2 = 3/4 u + 1/4 u1 + 1/4 dt L(u1); u3 = 1/3 u + 2/3 u2 + 2/3 dt L(u2)
        S.s[0] = {0, 0, 1, 0, 0, 0, -1, 0, -1, 0, 0};
        S.s[1] = {0.25, 0, 0.25, 0, 0, 0, 0, 1, -1, 0, 0};
        S.s[2] = {2.0 / 3.0, 0, 2.0 / 3.0, 0, 0, 0, 1, -1, -1, 0, 1};
        break;
    case 5: {  // SSP(5,4) of Spiteri & Ruuth (2002)
        const double b10 = 0.391752226571890;
        const double a21 = 0.555629506348765, b21 = 0.368410593050371;
        const double a32 = 0.379898148511597, b32 = 0.251891774271694;
        const double a43 = 0.821920045606868, b43 = 0.544974750228521;
        const double a52 = 0.517231671970585, a53 = 0.096059710526147, b53 = 0.063692468666290;
        const double a54 = 0.386708617503269, b54 = 0.226007483236906;
        S.s[0] = {0, 0, b10, 0, 0, 0, -1, 0, -1, 0, 0};          // delta1 -> D0
        S.s[1] = {a21, 0, b21, 0, 0, 0, 0, 1, -1, 0, 0};         // delta2 -> D1
        S.s[2] = {a32, 0, b32, 0, 0, 0, 1, 2, -1, 0, 0};         // delta3 -> D2 (delta2 kept in D1)
        S.s[3] = {a43, 0, b43, a53, a52, b53, 2, 0, 1, 1, 0};    // delta4 -> D0, X=D1 <- a52 d2 + a53 d3 + b53 dt L3
        S.s[4] = {a54, 1.0, b54, 0, 0, 0, 0, -1, 1, 0, 1};       // u^{n+1} = u^n + X + a54 d4 + b54 dt L4
        break;
    }
    default:
        S.stages = 0;
    }
    return S;
}

int auto_stages(int degree) { return degree + 1 <= 3 ? degree + 1 : 5; }

__global__ void to_f32_kernel(const double *__restrict__ a, float *__restrict__ b, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// total-degree basis: the caller's states hold only the modes l_x + l_y + l_z <= n (map[m] = their
// tensor index); internally every field of a cell keeps the full tensor layout with the other
// modes at zero.  rows = fields x cells; expand writes into a zeroed tensor array.
__global__ void td_expand_kernel(const double *__restrict__ src, double *__restrict__ dst, const int *map, int Mapi,
                                 int M, long long rows)
{
    const long long total = rows * Mapi;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / Mapi;
        dst[r * M + map[i - r * Mapi]] = src[i];
    }
}

__global__ void td_compact_kernel(const double *__restrict__ src, double *__restrict__ dst, const int *map, int Mapi,
                                  int M, long long rows)
{
    const long long total = rows * Mapi;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / Mapi;
        dst[i] = src[r * M + map[i - r * Mapi]];
    }
}

// dt from the per-block maxima of the prologue (Eq. timestep), or a fixed dt
__global__ void dt_kernel(const double *partial, int nblk, double fixed_dt, double cfl, double hmin, int P,
                          double *dtp, int advance, int *status)
{
    __shared__ double rc[256], rv[256];
    double c = 0.0, v = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        c = fmax(c, partial[2 * i]);
        v = fmax(v, partial[2 * i + 1]);
    }
    rc[threadIdx.x] = c;
    rv[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            rc[threadIdx.x] = fmax(rc[threadIdx.x], rc[threadIdx.x + s]);
            rv[threadIdx.x] = fmax(rv[threadIdx.x], rv[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double dt = fixed_dt > 0.0 ? fixed_dt : cfl * hmin / (2.0 * P * (rc[0] + rv[0]));
        if (!(dt > 0.0) || !isfinite(dt)) atomicOr(status, DG_STATUS_BADDT);
        if (advance) {
            dtp[0] = dt;
            dtp[1] += 1.0;
            dtp[2] += dt;
        } else {
            dtp[3] = dt;
        }
    }
}

// FP64 per-block partial sums of the cell means (fixed order => deterministic)
__global__ void sums_kernel(const double *U, long long ncell, int M, int nc, double *partial)
{
    __shared__ double red[256];
    for (int f = 0; f < nc; ++f) {
        double s = 0.0;
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ncell;
             k += (long long)gridDim.x * blockDim.x)
            s += U[((size_t)f * ncell + k) * M];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[blockIdx.x * nc + f] = red[0];
        __syncthreads();
    }
}

__global__ void sums_final_kernel(const double *partial, int nblk, int nc, double vol, double *out)
{
    if (threadIdx.x < nc) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partial[b * nc + threadIdx.x];
        out[threadIdx.x] = s * vol;
    }
}

// per-simulation time step of a batch: from the CFL maxima the first stage accumulated in
// descriptor.partial[0..1] (then reset for the next step), or a fixed dt
__global__ void batch_dt_kernel(const StageArgs *d, int nsims, int P, double fixed_dt)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsims; i += gridDim.x * blockDim.x) {
        const StageArgs &a = d[i];
        const double dt = fixed_dt > 0.0 ? fixed_dt : a.cfl * a.hmin / (2.0 * P * (a.partial[0] + a.partial[1]));
        if (!(dt > 0.0) || !isfinite(dt)) atomicOr(a.status, DG_STATUS_BADDT);
        double *dtp = const_cast<double *>(a.dtp);
        dtp[0] = dt;
        dtp[1] += 1.0;
        dtp[2] += dt;
        a.partial[0] = 0.0;
        a.partial[1] = 0.0;
    }
}

constexpr int kSumBlocks = 256;
constexpr int kMaxEvents = 12;
constexpr int kMaxStageGrid = 16384;  // persistent stage grid: SMs x resident CTAs (upper bound)

}  // namespace

struct dg_handle {
    dg_grid grid;
    int degree = 0;
    double gamma = 1.4, nu = 0.0, kappa = 0.0;
    dg_params p;
    int dim = 2, Q = 1, M = 1, nc = 4, nf = 4;
    long long ncell = 0;
    double h[3] = {1, 1, 1}, hmin = 1;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    Tables<double> td;
    Tables<float> tf;
    int stile[3], ptile[3], sgrid[3], pgrid[3];
    int pblocks = 0;

    double *U[2] = {nullptr, nullptr};
    float *Uhi[2] = {nullptr, nullptr};
    void *D[3] = {nullptr, nullptr, nullptr};
    int cur = 0;
    double *Sprev = nullptr, *wig = nullptr;
    double *dtp = nullptr;  // {dt, step, t, dt query}
    double *partial = nullptr;
    int partial_cap = 0;
    int fused_last = 0;  // the last enqueued step folded the prologue into its first stage
    int nev = 0;         // events recorded by the last timed step
    double *sums = nullptr;  // [kSumBlocks*nc] partials + [nc] result
    double *rhs_tmp = nullptr;
    int *status = nullptr;
    size_t nw = 0;

    cudaGraphExec_t graph = nullptr;
    double graph_dt = 0.0;

    // turbulence driving (Sec. 7.1)
    ForcingModes fm;
    double *fstate = nullptr;  // [kForceState] OU state
    double *smodes = nullptr;  // [kForceModes][6] projected, scaled amplitudes
    void *force = nullptr;     // Real [d][cell][node] driving acceleration
    void *ftab = nullptr;      // Real per-axis phase tables
    long long ftab_off[3] = {0, 0, 0};
    int forced_last = 0;  // the last enqueued step ran the driving kernels

    // total-degree basis (Sec. 2.3): modes seen by the caller, their tensor indices, staging buffer
    int Mapi = 1;
    // packed total-degree storage: the state arrays hold only the Mapi basis modes per cell (used where
    // the stage kernel reads and writes it: 3-D FP32-bulk, degrees 1 and 3, no tracer); Ms = stored
    // modes per cell, d_cmap[l] = stored index of tensor mode l or -1
    int packed = 0;
    int Ms = 1;
    int *d_cmap = nullptr;
    int *d_modemap = nullptr;
    double *stage = nullptr;  // [fields][cells][Mapi] for host transfers

    cudaEvent_t ev[kMaxEvents] = {nullptr};  // per-launch timing events of dg_step_timed

    std::string err;
};

namespace {

int fail(dg_t *h, int code, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

#define CK(h, call)                                                                             \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(h, DG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool fp32(const dg_t *h) { return h->p.precision == DG_FP32_BULK; }
size_t real_size(const dg_t *h) { return fp32(h) ? sizeof(float) : sizeof(double); }

void free_buffers(dg_t *h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    for (int i = 0; i < 2; ++i) {
        cudaFree(h->U[i]);
        cudaFree(h->Uhi[i]);
        h->U[i] = nullptr;
        h->Uhi[i] = nullptr;
    }
    for (int i = 0; i < 3; ++i) {
        cudaFree(h->D[i]);
        h->D[i] = nullptr;
    }
    cudaFree(h->Sprev);
    cudaFree(h->wig);
    cudaFree(h->dtp);
    cudaFree(h->partial);
    cudaFree(h->sums);
    cudaFree(h->rhs_tmp);
    cudaFree(h->status);
    h->Sprev = h->wig = h->dtp = h->partial = h->sums = h->rhs_tmp = nullptr;
    h->status = nullptr;
    cudaFree(h->fstate);
    cudaFree(h->smodes);
    cudaFree(h->force);
    cudaFree(h->ftab);
    h->fstate = h->smodes = nullptr;
    h->force = h->ftab = nullptr;
    cudaFree(h->d_modemap);
    cudaFree(h->d_cmap);
    cudaFree(h->stage);
    h->d_modemap = nullptr;
    h->d_cmap = nullptr;
    h->stage = nullptr;
}

bool total_degree(const dg_t *h) { return h->p.basis == DG_BASIS_TOTAL; }
// the caller's total-degree layout differs from the stored one (tensor storage with zeros)
bool expands(const dg_t *h) { return total_degree(h) && !h->packed; }
size_t nw_api(const dg_t *h) { return (size_t)h->nf * h->ncell * h->Mapi; }

int expand_state(dg_t *h, const double *src, double *dst)
{
    CK(h, cudaMemsetAsync(dst, 0, h->nw * sizeof(double), h->stream));
    td_expand_kernel<<<1024, 256, 0, h->stream>>>(src, dst, h->d_modemap, h->Mapi, h->M, (long long)h->nf * h->ncell);
    CK(h, cudaGetLastError());
    return DG_OK;
}

int compact_state(dg_t *h, const double *src, double *dst)
{
    td_compact_kernel<<<1024, 256, 0, h->stream>>>(src, dst, h->d_modemap, h->Mapi, h->M, (long long)h->nf * h->ncell);
    CK(h, cudaGetLastError());
    return DG_OK;
}

// driving buffers (allocated while forcing is on; the OU state starts with no update applied)
int alloc_forcing(dg_t *h)
{
    double L[3] = {1.0, 1.0, 1.0};
    for (int a = 0; a < h->dim; ++a) L[a] = h->grid.hi[a] - h->grid.lo[a];
    forcing_modes(h->dim, L, h->p.force_amp, &h->fm);
    if (h->force) return DG_OK;
    const size_t rs = real_size(h);
    long long ntab = 0;
    for (int a = 0; a < h->dim; ++a) ntab += (long long)h->grid.n[a] * h->Q * 10;
    std::vector<double> tab((size_t)ntab);
    forcing_phase_tables(h->dim, h->grid.n, L, h->degree, tab.data(), h->ftab_off);
    std::vector<float> tabf(fp32(h) ? (size_t)ntab : 0);
    for (size_t i = 0; i < tabf.size(); ++i) tabf[i] = (float)tab[i];
    const size_t nforce = (size_t)h->dim * h->ncell * h->M;
    if (cudaMalloc(&h->force, nforce * rs) != cudaSuccess || cudaMalloc(&h->ftab, (size_t)ntab * rs) != cudaSuccess ||
        cudaMalloc((void **)&h->fstate, kForceState * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&h->smodes, 6 * kForceModes * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->force);
        cudaFree(h->ftab);
        cudaFree(h->fstate);
        cudaFree(h->smodes);
        h->force = h->ftab = nullptr;
        h->fstate = h->smodes = nullptr;
        return fail(h, DG_ENOMEM, "driving buffers");
    }
    std::vector<double> f0(kForceState, 0.0);
    f0[0] = -1.0;
    CK(h, cudaMemcpy(h->ftab, fp32(h) ? (const void *)tabf.data() : (const void *)tab.data(), (size_t)ntab * rs,
                     cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->fstate, f0.data(), kForceState * sizeof(double), cudaMemcpyHostToDevice));
    CK(h, cudaMemset(h->smodes, 0, 6 * kForceModes * sizeof(double)));
    CK(h, cudaMemset(h->force, 0, nforce * rs));
    return DG_OK;
}

// driving acceleration at the volume nodes from the current amplitudes
cudaError_t launch_forcing_eval_any(const dg_t *h)
{
    return fp32(h) ? launch_forcing_eval_f32(h->dim, h->degree, h->grid.n, h->ncell, (const float *)h->ftab,
                                             h->ftab_off, h->smodes, (float *)h->force, h->stream)
                   : launch_forcing_eval_f64(h->dim, h->degree, h->grid.n, h->ncell, (const double *)h->ftab,
                                             h->ftab_off, h->smodes, (double *)h->force, h->stream);
}

int prepare_kernels(dg_t *h);

// Host-side fault injection for the failure paths of the allocations: with the environment
// variable DGX_FAULT=alloc:K, the K-th device allocation of every alloc_buffers call (K >= 1)
// fails as if cudaMalloc had reported cudaErrorMemoryAllocation, without calling it.  No device
// fault is involved; the caller sees DG_ENOMEM and a handle that owns no device memory.
int injected_alloc_failure()
{
    const char *f = getenv("DGX_FAULT");
    if (!f || strncmp(f, "alloc:", 6) != 0) return 0;
    const int k = atoi(f + 6);
    return k > 0 ? k : 0;
}

int alloc_buffers(dg_t *h)
{
    free_buffers(h);
    h->nc = h->dim + 2 + (h->p.tracer_on ? 1 : 0);
    h->nf = h->nc + (h->p.av_on ? 1 : 0);
    // modes seen by the caller: all tensor modes, or those with l_x + l_y + l_z <= n
    std::vector<int> modemap, cmap(h->M, -1);
    for (int t = 0; t < h->M; ++t) {
        const int lx = t % h->Q, ly = (t / h->Q) % h->Q, lz = h->dim == 3 ? t / (h->Q * h->Q) : 0;
        if (h->p.basis != DG_BASIS_TOTAL || lx + ly + lz <= h->degree) {
            cmap[t] = (int)modemap.size();
            modemap.push_back(t);
        }
    }
    h->Mapi = (int)modemap.size();
    h->packed = total_degree(h) && h->dim == 3 && fp32(h) && (h->degree == 1 || h->degree == 3) && !h->p.tracer_on;
    h->Ms = h->packed ? h->Mapi : h->M;
    h->nw = (size_t)h->nf * h->ncell * h->Ms;
    const size_t rs = real_size(h);
    const int fail_at = injected_alloc_failure();
    int nalloc = 0;
    auto al = [&](void **p, size_t bytes) -> int {
        if (++nalloc == fail_at)
            return fail(h, DG_ENOMEM, "cudaMalloc(%zu bytes): injected failure (DGX_FAULT=alloc:%d)", bytes, fail_at);
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, DG_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
        }
        return DG_OK;
    };
    int st = DG_OK;
    for (int i = 0; i < 2 && !st; ++i) st = al((void **)&h->U[i], h->nw * sizeof(double));
    if (fp32(h))
        for (int i = 0; i < 2 && !st; ++i) st = al((void **)&h->Uhi[i], h->nw * sizeof(float));
    for (int i = 0; i < 3 && !st; ++i) st = al(&h->D[i], h->nw * rs);
    if (!st) st = al((void **)&h->Sprev, h->ncell * sizeof(double));
    if (!st) st = al((void **)&h->wig, h->ncell * sizeof(double));
    if (!st) st = al((void **)&h->dtp, 4 * sizeof(double));
    int pt[3], sdummy[3];
    if (h->dim == 2) {
        if (fp32(h)) tiles_2d_f32(h->degree, h->p.tracer_on, sdummy, pt);
        else tiles_2d_f64(h->degree, h->p.tracer_on, sdummy, pt);
    } else {
        if (fp32(h)) tiles_3d_f32(h->degree, h->p.tracer_on, sdummy, pt);
        else tiles_3d_f64(h->degree, h->p.tracer_on, sdummy, pt);
    }
    for (int a = 0; a < 3; ++a) {
        h->stile[a] = sdummy[a];
        h->ptile[a] = pt[a];
        const int Na = a < h->dim ? h->grid.n[a] : 1;
        h->sgrid[a] = (Na + sdummy[a] - 1) / sdummy[a];
        h->pgrid[a] = (Na + pt[a] - 1) / pt[a];
    }
    h->pblocks = h->pgrid[0] * h->pgrid[1] * h->pgrid[2];
    h->partial_cap = h->pblocks > kMaxStageGrid ? h->pblocks : kMaxStageGrid;
    if (!st) st = al((void **)&h->partial, 2 * (size_t)h->partial_cap * sizeof(double));
    if (!st) st = al((void **)&h->sums, ((size_t)kSumBlocks * h->nc + h->nc) * sizeof(double));
    if (!st) st = al((void **)&h->status, sizeof(int));
    if (!st && h->packed) {
        st = al((void **)&h->d_cmap, cmap.size() * sizeof(int));
        if (!st && cudaMemcpy(h->d_cmap, cmap.data(), cmap.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(h, DG_ECUDA, "mode map upload");
    }
    if (!st && total_degree(h) && !h->packed) {
        st = al((void **)&h->d_modemap, modemap.size() * sizeof(int));
        if (!st) st = al((void **)&h->stage, nw_api(h) * sizeof(double));
        if (!st && cudaMemcpy(h->d_modemap, modemap.data(), modemap.size() * sizeof(int), cudaMemcpyHostToDevice) !=
                       cudaSuccess)
            st = fail(h, DG_ECUDA, "mode map upload");
    }
    if (st) {
        free_buffers(h);
        return st;
    }
    // zero state and auxiliary data
    for (int i = 0; i < 2; ++i) CK(h, cudaMemsetAsync(h->U[i], 0, h->nw * sizeof(double), h->stream));
    if (fp32(h))
        for (int i = 0; i < 2; ++i) CK(h, cudaMemsetAsync(h->Uhi[i], 0, h->nw * sizeof(float), h->stream));
    for (int i = 0; i < 3; ++i) CK(h, cudaMemsetAsync(h->D[i], 0, h->nw * rs, h->stream));
    CK(h, cudaMemsetAsync(h->Sprev, 0, h->ncell * sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->wig, 0, h->ncell * sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->dtp, 0, 4 * sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->cur = 0;
    if (h->p.forcing_on) {
        st = alloc_forcing(h);
        if (st) return st;
    }
    return prepare_kernels(h);
}

void base_stage_args(const dg_t *h, StageArgs &a)
{
    memset(&a, 0, sizeof a);
    for (int i = 0; i < 3; ++i) {
        a.N[i] = i < h->dim ? h->grid.n[i] : 1;
        a.bc[i] = i < h->dim ? h->grid.bc[i] : 0;
        a.ntile[i] = h->sgrid[i];
        a.h[i] = h->h[i];
    }
    a.hmin = h->hmin;
    a.gamma = h->gamma;
    a.nu = h->nu;
    a.kappa = h->kappa;
    a.ns_on = (h->nu > 0.0 || h->kappa > 0.0) ? 1 : 0;
    a.tracer_on = h->p.tracer_on;
    a.eta = h->p.tracer_eta;
    a.total_degree = total_degree(h) ? 1 : 0;
    a.cmap = h->packed ? h->d_cmap : nullptr;
    a.ms = h->Ms;
    a.av_on = h->p.av_on;
    a.av_scale = h->p.av_scale;
    a.f_v = h->p.f_v;
    a.f_tau = h->p.f_tau;
    a.nf = h->nf;
    a.ncell = h->ncell;
    a.wig = h->wig;
    a.dtp = h->dtp;
    a.status = h->status;
    a.force = h->p.forcing_on ? h->force : nullptr;
}

cudaError_t launch_stage_any(const dg_t *h, const StageArgs &a_in, int *grid = nullptr)
{
    StageArgs a = a_in;
    stage_consts(a, h->degree, h->dim);
    if (h->dim == 2)
        return fp32(h) ? launch_stage_2d_f32(h->degree, a, h->tf, h->stream, grid)
                       : launch_stage_2d_f64(h->degree, a, h->td, h->stream, grid);
    return fp32(h) ? launch_stage_3d_f32(h->degree, a, h->tf, h->stream, grid)
                   : launch_stage_3d_f64(h->degree, a, h->td, h->stream, grid);
}

cudaError_t launch_prologue_any(const dg_t *h, int update_sensor)
{
    PrologueArgs a;
    memset(&a, 0, sizeof a);
    for (int i = 0; i < 3; ++i) {
        a.N[i] = i < h->dim ? h->grid.n[i] : 1;
        a.ntile[i] = h->pgrid[i];
    }
    a.gamma = h->gamma;
    a.nf = h->nf;
    a.ncell = h->ncell;
    a.u = fp32(h) ? (const void *)h->Uhi[h->cur] : (const void *)h->U[h->cur];
    a.update_sensor = update_sensor && h->p.av_on;
    a.S_prev = h->Sprev;
    a.wig = h->wig;
    a.dtp = h->dtp;
    a.f_w = h->p.f_w;
    a.s_on = h->p.s_onset / ((double)(h->degree + 1) * (h->degree + 1));
    a.partial = h->partial;
    a.status = h->status;
    a.total_degree = total_degree(h) ? 1 : 0;
    a.cmap = h->packed ? h->d_cmap : nullptr;
    a.ms = h->Ms;
    if (h->dim == 2)
        return fp32(h) ? launch_prologue_2d_f32(h->degree, a, h->tf, h->stream)
                       : launch_prologue_2d_f64(h->degree, a, h->td, h->stream);
    return fp32(h) ? launch_prologue_3d_f32(h->degree, a, h->tf, h->stream)
                   : launch_prologue_3d_f64(h->degree, a, h->td, h->stream);
}

cudaError_t launch_limiter_any(const dg_t *h, const LimiterArgs &a)
{
    if (h->dim == 2)
        return fp32(h) ? launch_limiter_2d_f32(h->degree, a, h->tf, h->stream)
                       : launch_limiter_2d_f64(h->degree, a, h->td, h->stream);
    return fp32(h) ? launch_limiter_3d_f32(h->degree, a, h->tf, h->stream)
                   : launch_limiter_3d_f64(h->degree, a, h->td, h->stream);
}

// set the dynamic shared-memory attribute of this handle's kernels (launch with zero tiles)
int prepare_kernels(dg_t *h)
{
    StageArgs a;
    base_stage_args(h, a);
    a.ntile[0] = a.ntile[1] = a.ntile[2] = 0;
    CK(h, launch_stage_any(h, a));
    PrologueArgs pa;
    memset(&pa, 0, sizeof pa);
    if (h->dim == 2)
        CK(h, fp32(h) ? launch_prologue_2d_f32(h->degree, pa, h->tf, h->stream)
                      : launch_prologue_2d_f64(h->degree, pa, h->td, h->stream));
    else
        CK(h, fp32(h) ? launch_prologue_3d_f32(h->degree, pa, h->tf, h->stream)
                      : launch_prologue_3d_f64(h->degree, pa, h->td, h->stream));
    LimiterArgs la;
    memset(&la, 0, sizeof la);
    la.tracer_on = h->p.tracer_on;
    CK(h, launch_limiter_any(h, la));
    return DG_OK;
}

int stage_count(const dg_t *h) { return h->p.rk_stages > 0 ? h->p.rk_stages : auto_stages(h->degree); }

// arguments of stage i of a step that starts from the state buffer `c` (u^n), with or without
// the prologue folded into the first stage
void fill_stage_args(const dg_t *h, const Schedule &S, int i, int c, bool fused, StageArgs &a)
{
    const StageDesc &d = S.s[i];
    const int nx = 1 - c;
    base_stage_args(h, a);
    a.ubase = fp32(h) ? (const void *)h->Uhi[c] : (const void *)h->U[c];
    a.din = d.in >= 0 ? h->D[d.in] : nullptr;
    a.mode = d.last ? 2 : 1;
    a.xbuf = d.x >= 0 ? h->D[d.x] : nullptr;
    a.dout = d.out >= 0 ? h->D[d.out] : nullptr;
    a.ca = d.ca;
    a.cx = d.cx;
    a.cb = d.cb;
    a.za = d.za;
    a.zx = d.zx;
    a.zb = d.zb;
    a.write_z = d.write_z;
    a.uold = h->U[c];
    a.unew = h->U[nx];
    a.uhi_new = fp32(h) ? h->Uhi[nx] : nullptr;
    a.cfl = h->p.cfl;
    if (fused && i == 0) {
        a.fused = 1;
        a.partial = h->partial;
        a.S_prev = h->Sprev;
        a.wig_w = h->wig;
        a.f_w = h->p.f_w;
        a.s_on = h->p.s_onset / ((double)(h->degree + 1) * (h->degree + 1));
        a.epi_unit_dt = 1;  // delta_1 := L(u^n); scaled by cb dt where it is read
        a.cb = 1.0;
    }
    if (fused && i == 1) {
        a.din_dt = 1;
        a.din_coef = S.s[0].cb;
    }
}

// positivity limiter of the state entering a step (only initial data can need it: every later u^n
// is a limited stage output)
LimiterArgs entry_limiter_args(const dg_t *h)
{
    LimiterArgs la;
    memset(&la, 0, sizeof la);
    la.ncell = h->ncell;
    la.gamma = h->gamma;
    la.tracer_on = h->p.tracer_on;
    la.last = 1;
    la.ufull = h->U[h->cur];
    la.uhi = fp32(h) ? h->Uhi[h->cur] : nullptr;
    la.status = h->status;
    la.cmap = h->packed ? h->d_cmap : nullptr;
    la.ms = h->Ms;
    return la;
}

// positivity limiter after stage i of a step that starts from state buffer c
LimiterArgs stage_limiter_args(const dg_t *h, const Schedule &S, int i, int c)
{
    const StageDesc &d = S.s[i];
    const int nx = 1 - c;
    LimiterArgs la;
    memset(&la, 0, sizeof la);
    la.ncell = h->ncell;
    la.gamma = h->gamma;
    la.tracer_on = h->p.tracer_on;
    la.last = d.last;
    la.ubase = fp32(h) ? (const void *)h->Uhi[c] : (const void *)h->U[c];
    la.delta = d.last ? nullptr : h->D[d.out];
    la.ufull = d.last ? h->U[nx] : nullptr;
    la.uhi = d.last && fp32(h) ? h->Uhi[nx] : nullptr;
    la.status = h->status;
    la.cmap = h->packed ? h->d_cmap : nullptr;
    la.ms = h->Ms;
    return la;
}

// the separate step prologue (the path with the limiter, or one stage): limiter of the entering
// state, sensor + wiggle source + per-block CFL maxima, and the dt reduction -> dtp
int enqueue_prologue_dt(dg_t *h, double dt)
{
    if (h->p.positivity_on) CK(h, launch_limiter_any(h, entry_limiter_args(h)));
    CK(h, launch_prologue_any(h, 1));
    dt_kernel<<<1, 256, 0, h->stream>>>(h->partial, h->pblocks, dt > 0.0 ? dt : 0.0, h->p.cfl, h->hmin,
                                        h->degree + 1, h->dtp, 1, h->status);
    CK(h, cudaGetLastError());
    return DG_OK;
}

// enqueue one full step on h->stream (no host synchronisation).  With `ev`, an event is recorded
// before the first launch (ev[0]) and after each launch in launch order (ev[1..]).
//
// With two or more stages and no limiter, the step prologue (sensor, wiggle source, CFL speeds of
// u^n) is folded into the first stage kernel, which then stores L(u^n) unscaled because dt is not
// known yet; the second stage starts with the dt reduction of the first stage's per-CTA maxima
// and scales the stored first delta by its Runge-Kutta coefficient times dt.
int enqueue_step(dg_t *h, double dt, cudaEvent_t *ev = nullptr)
{
    const Schedule S = schedule_for(stage_count(h));
    if (!S.stages) return fail(h, DG_EINVAL, "unsupported Runge-Kutta stage count %d", stage_count(h));
    const bool fused = S.stages >= 2 && !h->p.positivity_on;
    int ne = 0;
    if (ev) CK(h, cudaEventRecord(ev[ne++], h->stream));
    if (h->p.forcing_on) {
        // driving updates due at the step's start time (device-resident t), then its field
        CK(h, launch_forcing_update(h->fm, h->dim, h->p.force_dt, h->p.force_ts, h->p.force_seed, 1, h->fstate,
                                    h->dtp + 2, h->smodes, h->status, h->stream));
        CK(h, launch_forcing_eval_any(h));
        if (ev) CK(h, cudaEventRecord(ev[ne++], h->stream));
    }
    if (!fused) {
        if (h->p.positivity_on) CK(h, launch_limiter_any(h, entry_limiter_args(h)));
        CK(h, launch_prologue_any(h, 1));
        if (ev) CK(h, cudaEventRecord(ev[ne++], h->stream));
        dt_kernel<<<1, 256, 0, h->stream>>>(h->partial, h->pblocks, dt > 0.0 ? dt : 0.0, h->p.cfl, h->hmin,
                                            h->degree + 1, h->dtp, 1, h->status);
        CK(h, cudaGetLastError());
        if (ev) CK(h, cudaEventRecord(ev[ne++], h->stream));
    }
    const int c = h->cur, nx = 1 - h->cur;
    int grid1 = 0;  // grid of the first stage: the number of per-CTA maxima the second reduces
    for (int i = 0; i < S.stages; ++i) {
        const StageDesc &d = S.s[i];
        StageArgs a;
        fill_stage_args(h, S, i, c, fused, a);
        if (fused && i == 1) {
            // the dt reduction runs at the start of the second stage
            a.dt_partial = h->partial;
            a.dt_nblk = grid1;
            a.dt_fixed = dt > 0.0 ? dt : 0.0;
        }
        int grid = 0;
        CK(h, launch_stage_any(h, a, &grid));
        if (h->p.positivity_on) CK(h, launch_limiter_any(h, stage_limiter_args(h, S, i, c)));
        if (ev) CK(h, cudaEventRecord(ev[ne++], h->stream));
        if (fused && i == 0) {
            if (grid > h->partial_cap) return fail(h, DG_EINVAL, "stage grid %d exceeds %d", grid, h->partial_cap);
            grid1 = grid;
        }
    }
    h->fused_last = fused ? 1 : 0;
    h->forced_last = h->p.forcing_on ? 1 : 0;
    h->nev = ne;
    h->cur = nx;
    return DG_OK;
}

int check_status(dg_t *h)
{
    int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (st) {
        CK(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (st & DG_STATUS_NONPHYS)
            return fail(h, DG_ENONPHYS, "non-physical state (rho <= 0 or p <= 0) at a quadrature point");
        if (st & DG_STATUS_FORCING)
            return fail(h, DG_EINVAL, "more than %lld driving updates due in one step (force_dt too small)",
                        kForceMaxUpdates);
        return fail(h, DG_ENONPHYS, "non-finite or non-positive time step");
    }
    return DG_OK;
}

int refresh_hi(dg_t *h)
{
    if (!fp32(h)) return DG_OK;
    to_f32_kernel<<<1024, 256, 0, h->stream>>>(h->U[h->cur], h->Uhi[h->cur], h->nw);
    CK(h, cudaGetLastError());
    return DG_OK;
}

// right-hand side in the internal (tensor) layout
int rhs_tensor(dg_t *h, double *dev_out)
{
    StageArgs a;
    base_stage_args(h, a);
    a.ubase = fp32(h) ? (const void *)h->Uhi[h->cur] : (const void *)h->U[h->cur];
    a.din = nullptr;
    a.mode = 0;
    a.rhs_out = dev_out;
    if (h->p.forcing_on) {
        // the field of the current driving state, without advancing it
        CK(h, launch_forcing_update(h->fm, h->dim, h->p.force_dt, h->p.force_ts, h->p.force_seed, 0, h->fstate,
                                    h->dtp + 2, h->smodes, h->status, h->stream));
        CK(h, launch_forcing_eval_any(h));
    }
    CK(h, launch_stage_any(h, a));
    return DG_OK;
}

int ensure_rhs_tmp(dg_t *h)
{
    if (h->rhs_tmp) return DG_OK;
    cudaError_t e = cudaMalloc((void **)&h->rhs_tmp, h->nw * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->rhs_tmp = nullptr;
        return fail(h, DG_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    return DG_OK;
}


}  // namespace

extern "C" {

const char *dg_status_string(int code)
{
    switch (code) {
    case DG_OK: return "ok";
    case DG_EINVAL: return "invalid argument";
    case DG_ENOMEM: return "out of device memory";
    case DG_ECUDA: return "CUDA error";
    case DG_ENONPHYS: return "non-physical state";
    case DG_ETIMEOUT: return "device wait timed out";
    case DG_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

int dg_default_params(dg_params *p)
{
    if (!p) return DG_EINVAL;
    p->precision = DG_FP64;
    p->rk_stages = 0;
    p->cfl = 0.5;
    p->av_on = 0;
    p->av_scale = 1.0;
    p->f_v = 2.5;
    p->f_tau = 0.5;
    p->f_w = 0.2;
    p->s_onset = 1e-4;
    p->positivity_on = 0;
    p->forcing_on = 0;
    p->force_amp = 0.0;
    p->force_ts = 1.0;
    p->force_dt = 0.01;
    p->force_seed = 0;
    p->tracer_on = 0;
    p->tracer_eta = 0.0;
    p->basis = DG_BASIS_TENSOR;
    return DG_OK;
}

int dg_create(const dg_grid *grid, int degree, double gamma, double nu, double kappa, dg_t **out)
{
    if (!out) return DG_EINVAL;
    *out = nullptr;
    if (!grid || grid->dim < 2 || grid->dim > 3 || degree < 0 || degree > kMaxDegree || !(gamma > 1.0) ||
        !(nu >= 0.0) || !(kappa >= 0.0))
        return DG_EINVAL;
    long long nc = 1;
    for (int a = 0; a < grid->dim; ++a) {
        if (grid->n[a] < 1 || !(grid->hi[a] > grid->lo[a]) || (grid->bc[a] != 0 && grid->bc[a] != 1))
            return DG_EINVAL;
        nc *= grid->n[a];
    }
    if (nc > 0x7fffffffLL) return DG_EINVAL;
    dg_t *h = new (std::nothrow) dg_t();
    if (!h) return DG_ENOMEM;
    h->grid = *grid;
    h->degree = degree;
    h->gamma = gamma;
    h->nu = nu;
    h->kappa = kappa;
    dg_default_params(&h->p);
    h->dim = grid->dim;
    h->Q = degree + 1;
    h->M = 1;
    for (int a = 0; a < h->dim; ++a) h->M *= h->Q;
    h->nc = h->dim + 2;
    h->ncell = nc;
    h->hmin = 1e300;
    for (int a = 0; a < h->dim; ++a) {
        h->h[a] = (grid->hi[a] - grid->lo[a]) / grid->n[a];
        if (h->h[a] < h->hmin) h->hmin = h->h[a];
    }
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return DG_ECUDA;
    }
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return DG_ECUDA;
    }
    make_tables(degree, &h->td, &h->tf);
    int st = alloc_buffers(h);
    if (st) {
        cudaStreamDestroy(h->cap_stream);
        delete h;
        return st;
    }
    *out = h;
    return DG_OK;
}

void dg_destroy(dg_t *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_buffers(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (int i = 0; i < kMaxEvents; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    delete h;
}

int dg_set_params(dg_t *h, const dg_params *p)
{
    if (!h || !p) return DG_EINVAL;
    if ((p->precision != DG_FP64 && p->precision != DG_FP32_BULK) || !(p->cfl > 0.0) ||
        (p->rk_stages != 0 && p->rk_stages != 1 && p->rk_stages != 2 && p->rk_stages != 3 && p->rk_stages != 5) ||
        (p->av_on != 0 && p->av_on != 1) || !(p->f_tau > 0.0) || p->av_scale < 0.0)
        return fail(h, DG_EINVAL, "invalid dg_params");
    if (p->positivity_on != 0 && p->positivity_on != 1) return fail(h, DG_EINVAL, "positivity_on must be 0 or 1");
    if ((p->forcing_on != 0 && p->forcing_on != 1) ||
        (p->forcing_on && (!(p->force_ts > 0.0) || !(p->force_dt > 0.0) || !(p->force_amp >= 0.0))))
        return fail(h, DG_EINVAL, "forcing needs force_ts > 0, force_dt > 0, force_amp >= 0");
    if ((p->tracer_on != 0 && p->tracer_on != 1) || !(p->tracer_eta >= 0.0))
        return fail(h, DG_EINVAL, "tracer_on must be 0 or 1 and tracer_eta >= 0");
    if (p->basis != DG_BASIS_TENSOR && p->basis != DG_BASIS_TOTAL) return fail(h, DG_EINVAL, "unknown basis");
    const bool realloc = p->precision != h->p.precision || p->av_on != h->p.av_on ||
                         p->tracer_on != h->p.tracer_on || p->basis != h->p.basis;
    h->p = *p;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (realloc) return alloc_buffers(h);
    if (h->p.forcing_on) return alloc_forcing(h);
    return DG_OK;
}

int dg_get_params(const dg_t *h, dg_params *p)
{
    if (!h || !p) return DG_EINVAL;
    *p = h->p;
    return DG_OK;
}

int dg_sizes(const dg_t *h, int *nfields, int *nmodes, long long *ncells)
{
    if (!h) return DG_EINVAL;
    if (nfields) *nfields = h->nf;
    if (nmodes) *nmodes = h->Mapi;
    if (ncells) *ncells = h->ncell;
    return DG_OK;
}

int dg_set_stream(dg_t *h, void *stream)
{
    if (!h) return DG_EINVAL;
    h->stream = (cudaStream_t)stream;
    return DG_OK;
}

int dg_set_state(dg_t *h, const double *host_w)
{
    if (!h || !host_w) return DG_EINVAL;
    if (expands(h)) {
        CK(h, cudaMemcpyAsync(h->stage, host_w, nw_api(h) * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        int st = expand_state(h, h->stage, h->U[h->cur]);
        if (st) return st;
    } else {
        CK(h, cudaMemcpyAsync(h->U[h->cur], host_w, h->nw * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    int st = refresh_hi(h);
    if (st) return st;
    CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

int dg_set_state_device(dg_t *h, const double *dev_w)
{
    if (!h || !dev_w) return DG_EINVAL;
    if (expands(h)) {
        int st = expand_state(h, dev_w, h->U[h->cur]);
        if (st) return st;
    } else {
        CK(h, cudaMemcpyAsync(h->U[h->cur], dev_w, h->nw * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    return refresh_hi(h);
}

int dg_get_state(dg_t *h, double *host_w)
{
    if (!h || !host_w) return DG_EINVAL;
    if (expands(h)) {
        int st = compact_state(h, h->U[h->cur], h->stage);
        if (st) return st;
        CK(h, cudaMemcpyAsync(host_w, h->stage, nw_api(h) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    } else {
        CK(h, cudaMemcpyAsync(host_w, h->U[h->cur], h->nw * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    return check_status(h);
}

int dg_get_state_device(dg_t *h, double *dev_w)
{
    if (!h || !dev_w) return DG_EINVAL;
    if (expands(h)) return compact_state(h, h->U[h->cur], dev_w);
    CK(h, cudaMemcpyAsync(dev_w, h->U[h->cur], h->nw * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    return DG_OK;
}


int dg_rhs_device(dg_t *h, double *dev_out)
{
    if (!h || !dev_out) return DG_EINVAL;
    if (!expands(h)) return rhs_tensor(h, dev_out);
    int st = ensure_rhs_tmp(h);
    if (!st) st = rhs_tensor(h, h->rhs_tmp);
    if (!st) st = compact_state(h, h->rhs_tmp, dev_out);
    return st;
}

int dg_rhs(dg_t *h, double *host_out)
{
    if (!h || !host_out) return DG_EINVAL;
    int st = ensure_rhs_tmp(h);
    if (!st) st = rhs_tensor(h, h->rhs_tmp);
    if (st) return st;
    if (expands(h)) {
        st = compact_state(h, h->rhs_tmp, h->stage);
        if (st) return st;
        CK(h, cudaMemcpyAsync(host_out, h->stage, nw_api(h) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    } else {
        CK(h, cudaMemcpyAsync(host_out, h->rhs_tmp, h->nw * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    return check_status(h);
}

int dg_step(dg_t *h, double dt)
{
    if (!h) return DG_EINVAL;
    return enqueue_step(h, dt);
}

int dg_steps(dg_t *h, int nsteps, double dt)
{
    if (!h || nsteps < 0) return DG_EINVAL;
    int done = 0;
    if (h->cur != 0 && nsteps > 0) {  // bring the ping-pong parity back to 0
        int st = enqueue_step(h, dt);
        if (st) return st;
        ++done;
    }
    if (nsteps - done >= 2) {
        if (!h->graph || h->graph_dt != dt) {
            if (h->graph) cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
            cudaStream_t user = h->stream;
            h->stream = h->cap_stream;
            CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            int st = enqueue_step(h, dt);
            if (!st) st = enqueue_step(h, dt);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
            h->stream = user;
            if (st) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return fail(h, DG_ECUDA, "graph capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&h->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                h->graph = nullptr;
                return fail(h, DG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
            }
            h->graph_dt = dt;
        }
        while (nsteps - done >= 2) {
            CK(h, cudaGraphLaunch(h->graph, h->stream));
            done += 2;
        }
    }
    while (done < nsteps) {
        int st = enqueue_step(h, dt);
        if (st) return st;
        ++done;
    }
    return DG_OK;
}

int dg_step_timed(dg_t *h, double dt, float *ms, int nms)
{
    if (!h || !ms) return DG_EINVAL;
    const int ns = stage_count(h);
    const int nl = 2 + ns;
    if (nms < nl) return fail(h, DG_EINVAL, "dg_step_timed needs room for %d launch times", nl);
    for (int i = 0; i < kMaxEvents; ++i)
        if (!h->ev[i]) CK(h, cudaEventCreate(&h->ev[i]));
    int st = enqueue_step(h, dt, h->ev);
    if (st) return st;
    CK(h, cudaEventSynchronize(h->ev[h->nev - 1]));
    float d[kMaxEvents];
    for (int i = 0; i + 1 < h->nev; ++i) CK(h, cudaEventElapsedTime(&d[i], h->ev[i], h->ev[i + 1]));
    // the driving kernels (if any) run first; their time is counted with the step prologue
    const int o = h->forced_last ? 1 : 0;
    const float fms = h->forced_last ? d[0] : 0.0f;
    if (h->fused_last) {
        // launch order: stage 1 (with the prologue work), stages 2..s (the second starts with the
        // dt reduction, so there is no separate dt launch)
        ms[0] = fms;
        ms[1] = 0.0f;
        for (int i = 0; i < ns; ++i) ms[2 + i] = d[o + i];
    } else {
        for (int i = 0; i < nl; ++i) ms[i] = d[o + i];
        ms[0] += fms;
    }
    return DG_OK;
}

int dg_sync(dg_t *h)
{
    if (!h) return DG_EINVAL;
    return check_status(h);
}

int dg_max_dt(dg_t *h, double *dt)
{
    if (!h || !dt) return DG_EINVAL;
    CK(h, launch_prologue_any(h, 0));
    dt_kernel<<<1, 256, 0, h->stream>>>(h->partial, h->pblocks, 0.0, h->p.cfl, h->hmin, h->degree + 1, h->dtp, 0,
                                        h->status);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(dt, h->dtp + 3, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return check_status(h);
}

int dg_conserved_sums(dg_t *h, double *out)
{
    if (!h || !out) return DG_EINVAL;
    double vol = 1.0;
    for (int a = 0; a < h->dim; ++a) vol *= h->h[a];
    sums_kernel<<<kSumBlocks, 256, 0, h->stream>>>(h->U[h->cur], h->ncell, h->Ms, h->nc, h->sums);
    sums_final_kernel<<<1, 32, 0, h->stream>>>(h->sums, kSumBlocks, h->nc, vol, h->sums + kSumBlocks * h->nc);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(out, h->sums + kSumBlocks * h->nc, h->nc * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

int dg_get_aux(dg_t *h, double *S_prev, double *wig, double *scal)
{
    if (!h) return DG_EINVAL;
    if (S_prev)
        CK(h, cudaMemcpyAsync(S_prev, h->Sprev, h->ncell * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (wig) CK(h, cudaMemcpyAsync(wig, h->wig, h->ncell * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (scal) CK(h, cudaMemcpyAsync(scal, h->dtp, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

int dg_set_aux(dg_t *h, const double *S_prev, const double *wig, const double *scal)
{
    if (!h) return DG_EINVAL;
    if (S_prev)
        CK(h, cudaMemcpyAsync(h->Sprev, S_prev, h->ncell * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (wig) CK(h, cudaMemcpyAsync(h->wig, wig, h->ncell * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (scal) CK(h, cudaMemcpyAsync(h->dtp, scal, 3 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

int dg_get_forcing(dg_t *h, double *host_state)
{
    if (!h || !host_state) return DG_EINVAL;
    if (!h->p.forcing_on || !h->fstate) return fail(h, DG_EINVAL, "forcing is off");
    CK(h, cudaMemcpyAsync(host_state, h->fstate, kForceState * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return check_status(h);
}

int dg_set_forcing(dg_t *h, const double *host_state)
{
    if (!h || !host_state) return DG_EINVAL;
    if (!h->p.forcing_on || !h->fstate) return fail(h, DG_EINVAL, "forcing is off");
    CK(h, cudaMemcpyAsync(h->fstate, host_state, kForceState * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
}

const char *dg_last_error(const dg_t *h)
{
    if (!h) return "null handle";
    return h->err.c_str();
}


}  // extern "C"

// ------------------------------------------------------------------ batched ensembles

struct dg_batch {
    struct Group {
        int dim = 2, degree = 0, prec = 0, av = 0, ns = 0, stages = 0;
        int lim = 0;  // positivity limiter: separate step prologue per member, limiter after every stage
        std::vector<int> members;
        int total_tiles = 0;
        StageArgs *d_desc = nullptr;  // [2 parities][stages][members]
        int *d_off = nullptr;         // [members + 1] tile prefix sums
        double *d_max = nullptr;      // [members][2] CFL maxima of the first stage
        const dg_t *rep = nullptr;    // member that owns the group's operator tables
        cudaStream_t st = nullptr;
        cudaEvent_t done = nullptr;
    };
    std::vector<dg_t *> sims;
    std::vector<Group> groups;
    cudaStream_t stream = nullptr;  // stream of the members (the batch's origin stream)
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph = nullptr;
    double graph_dt = 0.0;
    int parity = 0;
    std::string err;
};

namespace {

int bfail(dg_batch_t *b, int code, const char *msg)
{
    if (b) b->err = msg;
    return code;
}

// one batched stage launch of a group; prepare_only sets the kernel attributes without launching
cudaError_t launch_batch_group(const dg_batch::Group &g, int parity, int i, cudaStream_t s, bool prepare_only = false)
{
    const StageArgs *d = g.d_desc + ((size_t)parity * g.stages + i) * g.members.size();
    const int nm = (int)g.members.size();
    const int tot = prepare_only ? 0 : g.total_tiles;
    if (g.dim == 2)
        return g.prec ? launch_stage_batch_2d_f32(g.degree, g.av, g.ns, d, g.d_off, nm, tot, g.rep->tf, s)
                      : launch_stage_batch_2d_f64(g.degree, g.av, g.ns, d, g.d_off, nm, tot, g.rep->td, s);
    return g.prec ? launch_stage_batch_3d_f32(g.degree, g.av, g.ns, d, g.d_off, nm, tot, g.rep->tf, s)
                  : launch_stage_batch_3d_f64(g.degree, g.av, g.ns, d, g.d_off, nm, tot, g.rep->td, s);
}

// one step of every member: each group on its own stream, forked from and joined to `origin`
int enqueue_batch_step(dg_batch_t *b, double dt, cudaStream_t origin)
{
    if (cudaEventRecord(b->fork, origin) != cudaSuccess) return bfail(b, DG_ECUDA, "cudaEventRecord");
    for (auto &g : b->groups) {
        if (cudaStreamWaitEvent(g.st, b->fork, 0) != cudaSuccess) return bfail(b, DG_ECUDA, "cudaStreamWaitEvent");
        // members of a limiter group issue their own prologue and limiter launches on the group's stream
        auto on_group_stream = [&](dg_t *h, auto fn) -> int {
            cudaStream_t own = h->stream;
            h->stream = g.st;
            const int r = fn(h);
            h->stream = own;
            return r;
        };
        if (g.lim) {
            for (int m : g.members) {
                dg_t *h = b->sims[m];
                if (on_group_stream(h, [&](dg_t *hh) { return enqueue_prologue_dt(hh, dt); }))
                    return bfail(b, DG_ECUDA, h->err.c_str());
            }
        }
        const Schedule S = schedule_for(g.stages);
        for (int i = 0; i < g.stages; ++i) {
            if (launch_batch_group(g, b->parity, i, g.st) != cudaSuccess) return bfail(b, DG_ECUDA, "batched stage launch");
            if (g.lim) {
                for (int m : g.members) {
                    dg_t *h = b->sims[m];
                    const int r = on_group_stream(h, [&](dg_t *hh) -> int {
                        CK(hh, launch_limiter_any(hh, stage_limiter_args(hh, S, i, b->parity)));
                        return DG_OK;
                    });
                    if (r) return bfail(b, DG_ECUDA, "member limiter launch");
                }
                continue;
            }
            if (i == 0) {
                const StageArgs *d = g.d_desc + (size_t)b->parity * g.stages * g.members.size();
                batch_dt_kernel<<<1, 256, 0, g.st>>>(d, (int)g.members.size(), g.degree + 1, dt > 0.0 ? dt : 0.0);
                if (cudaGetLastError() != cudaSuccess) return bfail(b, DG_ECUDA, "batched dt launch");
            }
        }
        if (cudaEventRecord(g.done, g.st) != cudaSuccess) return bfail(b, DG_ECUDA, "cudaEventRecord");
        if (cudaStreamWaitEvent(origin, g.done, 0) != cudaSuccess) return bfail(b, DG_ECUDA, "cudaStreamWaitEvent");
    }
    b->parity ^= 1;
    for (dg_t *h : b->sims) h->cur ^= 1;
    return DG_OK;
}

void free_batch(dg_batch_t *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto &g : b->groups) {
        cudaFree(g.d_desc);
        cudaFree(g.d_off);
        cudaFree(g.d_max);
        if (g.st) cudaStreamDestroy(g.st);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->fork) cudaEventDestroy(b->fork);
}

}  // namespace

extern "C" {

int dg_batch_create(dg_t *const *sims, int count, dg_batch_t **out)
{
    if (!out || !sims || count < 1) return DG_EINVAL;
    *out = nullptr;
    for (int k = 0; k < count; ++k) {
        const dg_t *h = sims[k];
        if (!h) return DG_EINVAL;
        // driving and tracer members, and members in packed total-degree storage (the batched kernel
        // reads tensor storage), are not batched
        if (h->p.forcing_on || h->p.tracer_on || h->packed || stage_count(h) < 2) return DG_EUNSUPPORTED;
        if (h->cur != sims[0]->cur || h->device != sims[0]->device || h->stream != sims[0]->stream)
            return DG_EINVAL;
    }
    dg_batch_t *b = new (std::nothrow) dg_batch_t();
    if (!b) return DG_ENOMEM;
    b->sims.assign(sims, sims + count);
    b->stream = sims[0]->stream;
    b->parity = sims[0]->cur;
    std::map<std::tuple<int, int, int, int, int, int>, int> key_to_group;
    for (int k = 0; k < count; ++k) {
        const dg_t *h = sims[k];
        const int ns = (h->nu > 0.0 || h->kappa > 0.0) ? 1 : 0;
        const auto key = std::make_tuple(h->dim, h->degree, (int)fp32(h), h->p.av_on, ns, h->p.positivity_on);
        auto it = key_to_group.find(key);
        if (it == key_to_group.end()) {
            dg_batch::Group g;
            g.dim = h->dim;
            g.degree = h->degree;
            g.prec = fp32(h) ? 1 : 0;
            g.av = h->p.av_on;
            g.ns = ns;
            g.stages = stage_count(h);
            g.lim = h->p.positivity_on;
            g.rep = h;
            it = key_to_group.emplace(key, (int)b->groups.size()).first;
            b->groups.push_back(g);
        }
        b->groups[it->second].members.push_back(k);
    }
    int st = DG_OK;
    for (auto &g : b->groups) {
        const int nm = (int)g.members.size();
        const Schedule S = schedule_for(g.stages);
        std::vector<int> off(nm + 1, 0);
        for (int m = 0; m < nm; ++m) {
            const dg_t *h = sims[g.members[m]];
            off[m + 1] = off[m] + h->sgrid[0] * h->sgrid[1] * h->sgrid[2];
        }
        g.total_tiles = off[nm];
        if (cudaMalloc((void **)&g.d_off, sizeof(int) * (nm + 1)) != cudaSuccess ||
            cudaMalloc((void **)&g.d_max, sizeof(double) * 2 * nm) != cudaSuccess ||
            cudaMalloc((void **)&g.d_desc, sizeof(StageArgs) * 2 * g.stages * nm) != cudaSuccess) {
            cudaGetLastError();
            st = DG_ENOMEM;
            break;
        }
        std::vector<StageArgs> host((size_t)2 * g.stages * nm);
        for (int par = 0; par < 2; ++par)
            for (int i = 0; i < g.stages; ++i)
                for (int m = 0; m < nm; ++m) {
                    StageArgs &a = host[((size_t)par * g.stages + i) * nm + m];
                    // without the limiter the step prologue is folded into the first stage; with it the
                    // members run the separate prologue and the stages read each member's dt
                    fill_stage_args(sims[g.members[m]], S, i, par, !g.lim, a);
                    if (i == 0 && !g.lim) a.partial = g.d_max + 2 * m;  // per-simulation maxima (atomics)
                    stage_consts(a, g.degree, g.dim);
                }
        if (cudaMemcpy(g.d_off, off.data(), sizeof(int) * (nm + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(g.d_max, 0, sizeof(double) * 2 * nm) != cudaSuccess ||
            cudaMemcpy(g.d_desc, host.data(), sizeof(StageArgs) * host.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            st = DG_ECUDA;
            break;
        }
        // kernel attributes and occupancy, before any capture
        if (launch_batch_group(g, 0, 0, g.st, true) != cudaSuccess) {
            st = DG_ECUDA;
            break;
        }
    }
    if (!st && (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        st = DG_ECUDA;
    }
    if (st) {
        free_batch(b);
        delete b;
        return st;
    }
    *out = b;
    return DG_OK;
}

int dg_batch_step(dg_batch_t *b, int nsteps, double dt)
{
    if (!b || nsteps < 0) return DG_EINVAL;
    int done = 0;
    if (b->parity != 0 && nsteps > 0) {
        int st = enqueue_batch_step(b, dt, b->stream);
        if (st) return st;
        ++done;
    }
    if (nsteps - done >= 2) {
        if (!b->graph || b->graph_dt != dt) {
            if (b->graph) cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return bfail(b, DG_ECUDA, "cudaStreamBeginCapture");
            int st = enqueue_batch_step(b, dt, b->cap);
            if (!st) st = enqueue_batch_step(b, dt, b->cap);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
            if (st) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return bfail(b, DG_ECUDA, "graph capture");
            const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                b->graph = nullptr;
                return bfail(b, DG_ECUDA, "graph instantiate");
            }
            b->graph_dt = dt;
        }
        while (nsteps - done >= 2) {
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return bfail(b, DG_ECUDA, "cudaGraphLaunch");
            done += 2;
        }
    }
    while (done < nsteps) {
        int st = enqueue_batch_step(b, dt, b->stream);
        if (st) return st;
        ++done;
    }
    return DG_OK;
}

int dg_batch_sync(dg_batch_t *b)
{
    if (!b) return DG_EINVAL;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, DG_ECUDA, "cudaStreamSynchronize");
    int worst = DG_OK;
    for (dg_t *h : b->sims) {
        const int st = check_status(h);
        if (st && !worst) worst = st;
    }
    if (worst) b->err = "a member reported a non-physical state or time step";
    return worst;
}

const char *dg_batch_last_error(const dg_batch_t *b) { return b ? b->err.c_str() : "null batch"; }

void dg_batch_destroy(dg_batch_t *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
}

}  // extern "C"
