// Internal declarations shared by the host API (dgx_api.cu) and the kernel
// instantiation units (dgx_inst_*.cu).  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace dgx {

// Launch set-up of one kernel, done once per device: cudaFuncSetAttribute applies to the current
// device only, so a process that uses several GPUs needs the dynamic shared-memory attribute set
// on each of them before the first launch there.  Also records the device's SM count and the
// resident CTAs per SM of the kernel at (threads, smem).  The first launch on a device does the
// set-up; handles and batches make that launch at creation (a launch over zero tiles), so it never
// falls inside a stream capture.  Thread-safe.
constexpr int kMaxDevices = 64;
struct KernelSetup {
    std::mutex m;
    bool done[kMaxDevices] = {};
    int sms[kMaxDevices] = {};
    int blocks_per_sm[kMaxDevices] = {};
};

template <typename K>
cudaError_t kernel_setup(KernelSetup &ks, K kernel, int threads, size_t smem, int *sms = nullptr,
                         int *blocks_per_sm = nullptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(ks.m);
    if (!ks.done[dev]) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&ks.sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ks.blocks_per_sm[dev], kernel, threads, smem);
        if (e != cudaSuccess) return e;
        if (ks.blocks_per_sm[dev] < 1) ks.blocks_per_sm[dev] = 1;
        ks.done[dev] = true;
    }
    if (sms) *sms = ks.sms[dev];
    if (blocks_per_sm) *blocks_per_sm = ks.blocks_per_sm[dev];
    return cudaSuccess;
}

constexpr int kMaxDegree = 5;
// bits of the device status word
constexpr int DG_STATUS_NONPHYS = 1;  // rho <= 0, p <= 0 or non-finite value at a quadrature point
constexpr int DG_STATUS_BADDT = 2;    // non-finite or non-positive CFL time step
constexpr int DG_STATUS_FORCING = 4;  // more driving updates due in one step than the kernel applies
constexpr int kMaxQ = kMaxDegree + 1;

// Per-degree operator tables, host-generated in long double (dgx_tables.cu):
//   B[i][m]  = Pt_m(x_i)                modal -> nodal (collocation at Gauss points)
//   Dn[i][m] = l'_m(x_i)                nodal derivative on [-1,1]
//   Wd[i][m] = g_m Dn[m][i]             transposed, Gauss-weighted derivative (weak divergence)
//   G[i]     = g_i                      Gauss weights
//   Lp[m], Lm[m] = l_m(+1), l_m(-1)     traces of the nodal Lagrange basis
//   Cm[m], Cp[m]  recovered value at the interface from the left / right cell's nodal line
//   Dm[m], Dp[m]  recovered normal derivative (multiply by 1/(f h)) from left / right cell
// All indices run over Q = n+1 entries; arrays are sized for the largest degree.
template <typename Real>
struct Tables {
    Real B[kMaxQ][kMaxQ];
    Real Dn[kMaxQ][kMaxQ];
    Real Wd[kMaxQ][kMaxQ];
    Real G[kMaxQ];
    Real Lp[kMaxQ], Lm[kMaxQ];
    Real Cm[kMaxQ], Cp[kMaxQ];
    Real Dm[kMaxQ], Dp[kMaxQ];
    Real inv_f;  // 1/f, f the recovery overlap fraction
};

void make_tables(int degree, Tables<double> *td, Tables<float> *tf);

// Arguments of the fused right-hand-side / Runge-Kutta stage kernel.
// indices of StageArgs::kf / kd
enum StageConst {
    SK_TWO_H = 0,   // 2 / h_a, a = 0..2
    SK_INV_H = 3,   // 1 / h_a
    SK_CAX = 6,     // face-integral weight of axis a over h_a (1/2 in 2-D, 1/4 in 3-D)
    SK_EPS = 9,     // av_scale h_min / (n+1): AV viscosity per unit alpha c_s
    SK_INV_TAU,     // (n+1) / (f_tau h_min): alpha decay rate per unit c_s
    SK_FV,
    SK_GAMMA,
    SK_NU,
    SK_KAPPA,
    SK_ETA,         // tracer diffusivity (Sec. 3.4)
    SK_CA, SK_CX, SK_CB, SK_ZA, SK_ZX, SK_ZB,  // Runge-Kutta register coefficients
    SK_COUNT
};

struct StageArgs {
    int N[3];      // cells per axis (1 for unused axes)
    int bc[3];     // 0 periodic, 1 outflow
    int ntile[3];  // tiles per axis (the z-marching kernel: columns along x, y and chunks along z)
    int zchunk;    // z-marching kernel: planes per chunk
    int reserved_;
    double h[3];
    double hmin;
    double gamma, nu, kappa;
    int ns_on;  // nu > 0 or kappa > 0
    int tracer_on;  // passive tracer field rho c after the energy (Sec. 3.4)
    double eta;     // its diffusivity
    int total_degree;  // basis of modes l_x + l_y + l_z <= n (Sec. 2.3): the others are kept at zero
    // packed total-degree storage: the state arrays hold ms modes per cell, the total-degree modes
    // in tensor order; cmap[l] = stored index of tensor mode l, or -1 (null: tensor storage, ms = NP)
    const int *cmap;
    int ms;
    int av_on;
    double av_scale, f_v, f_tau;
    int nf;  // fields incl. alpha
    long long ncell;

    // stage input state = ubase + din (din may be null: delta = 0)
    const void *ubase;  // Real*: FP32 high copy of u^n (bulk) or u^n itself (FP64)
    const void *din;    // Real*
    const double *wig;  // per cell wiggle source
    const void *force;  // Real* driving acceleration at the volume nodes [d][cell][node], or null
    const double *dtp;  // device scalars {dt, step, t}

    // epilogue
    int mode;  // 0: write L to rhs_out; 1: delta stage; 2: last stage (commit u^{n+1})
    double *rhs_out;
    void *xbuf;  // Real*: auxiliary register read (cx, zx) and written (write_z)
    void *dout;  // Real*
    double ca, cx, cb, za, zx, zb;
    int write_z;
    const double *uold;  // FP64 u^n
    double *unew;        // FP64 u^{n+1}
    float *uhi_new;      // FP32 copy of u^{n+1} (bulk mode) or null

    int *status;

    // first stage of a step with the prologue folded in: sensor + wiggle source per cell and
    // per-CTA maxima of c_s and |v| of u^n; the stage stores L(u^n) itself (dt not yet known)
    int fused;
    double *partial;   // [gridDim.x][2]
    double *S_prev;    // sensor history (read, then updated)
    double *wig_w;     // wiggle source (written)
    double f_w, s_on;
    int epi_unit_dt;   // epilogue uses dt = 1 (delta_out = L when cb = 1)
    // the stored input delta is din_coef * dt times the true one's 1/(din_coef dt)-scaled value:
    // true delta = din_coef * dtp[0] * din when din_dt is set
    int din_dt;
    double din_coef;
    double cfl;  // CFL factor (read by the batched time-step kernel)
    // second stage of a step with the prologue folded in: every CTA computes the step's dt from
    // the first stage's per-CTA maxima dt_partial[dt_nblk][2] (or takes dt_fixed > 0); CTA 0
    // publishes it to dtp {dt, step + 1, t + dt}
    const double *dt_partial;
    int dt_nblk;
    double dt_fixed;

    // per-simulation constants of the stage body in both precisions, derived on the host from the
    // fields above by stage_consts() (FP64 divisions inside the tile loop are costly on this part)
    float kf[SK_COUNT];
    double kd[SK_COUNT];
};

static_assert(sizeof(StageArgs) % 8 == 0 && alignof(StageArgs) == 8, "StageArgs is copied as 8-byte words");

// fill StageArgs::kf / kd (degree: polynomial degree, dim: 2 or 3); call after every other field is set
inline void stage_consts(StageArgs &a, int degree, int dim)
{
    double k[SK_COUNT];
    for (int i = 0; i < 3; ++i) {
        k[SK_TWO_H + i] = 2.0 / a.h[i];
        k[SK_INV_H + i] = 1.0 / a.h[i];
        k[SK_CAX + i] = (dim == 2 ? 0.5 : 0.25) / a.h[i];
    }
    k[SK_EPS] = a.av_scale * a.hmin / (degree + 1);
    k[SK_INV_TAU] = (degree + 1) / (a.f_tau * a.hmin);
    k[SK_FV] = a.f_v;
    k[SK_GAMMA] = a.gamma;
    k[SK_NU] = a.nu;
    k[SK_KAPPA] = a.kappa;
    k[SK_ETA] = a.eta;
    k[SK_CA] = a.ca;
    k[SK_CX] = a.cx;
    k[SK_CB] = a.cb;
    k[SK_ZA] = a.za;
    k[SK_ZX] = a.zx;
    k[SK_ZB] = a.zb;
    for (int i = 0; i < SK_COUNT; ++i) {
        a.kd[i] = k[i];
        a.kf[i] = (float)k[i];
    }
}

// Arguments of the step-prologue kernel (CFL speeds + oscillation sensor).
struct PrologueArgs {
    int N[3];
    int ntile[3];
    double gamma;
    int nf;
    long long ncell;
    const void *u;  // Real*
    int update_sensor;
    double *S_prev;
    double *wig;
    const double *dtp;
    double f_w, s_on;
    double *partial;  // [blocks][2] max c_s, max |v|
    int *status;
    int total_degree;  // sensor: high modes are l_x + l_y + l_z = n instead of some l_a = n
    const int *cmap;   // packed total-degree storage (see StageArgs::cmap), or null
    int ms;            // stored modes per cell
};

// Arguments of the positivity-limiter kernel (Sec. 4.2), run after a stage.
struct LimiterArgs {
    long long ncell;
    double gamma;
    int last;            // 1: limit u^{n+1} (FP64 u, plus the FP32 copy in bulk mode); 0: u_base + delta
    const void *ubase;   // Real*: stage base (u_hi in bulk mode, u^n in FP64)
    void *delta;         // Real*: stage delta, limited in place
    double *ufull;       // FP64 state, limited in place (last stage)
    float *uhi;          // FP32 copy of ufull to refresh (bulk mode, last stage) or null
    int *status;
    int tracer_on;       // a passive tracer follows the energy: d+3 conserved fields are scaled
    const int *cmap;     // packed total-degree storage (see StageArgs::cmap), or null
    int ms;              // stored modes per cell
};

struct LaunchCfg {
    int blocks;
    int threads;
    size_t smem;
};

// Kernel launchers (defined in the instantiation units).  `prec` 0 = FP64, 1 = FP32.
cudaError_t launch_stage(int dim, int degree, int prec, const StageArgs &a, const Tables<double> &td,
                         const Tables<float> &tf, cudaStream_t s);
cudaError_t launch_prologue(int dim, int degree, int prec, const PrologueArgs &a, const Tables<double> &td,
                            const Tables<float> &tf, cudaStream_t s, int *nblocks_out);
void stage_tiles(int dim, int degree, int prec, int tile[3]);
void prologue_tiles(int dim, int degree, int prec, int tile[3]);

cudaError_t launch_stage_2d_f64(int degree, const StageArgs &a, const Tables<double> &t, cudaStream_t s, int *grid);
cudaError_t launch_stage_2d_f32(int degree, const StageArgs &a, const Tables<float> &t, cudaStream_t s, int *grid);
cudaError_t launch_stage_3d_f64(int degree, const StageArgs &a, const Tables<double> &t, cudaStream_t s, int *grid);
cudaError_t launch_stage_3d_f32(int degree, const StageArgs &a, const Tables<float> &t, cudaStream_t s, int *grid);
cudaError_t launch_prologue_2d_f64(int degree, const PrologueArgs &a, const Tables<double> &t, cudaStream_t s);
cudaError_t launch_prologue_2d_f32(int degree, const PrologueArgs &a, const Tables<float> &t, cudaStream_t s);
cudaError_t launch_prologue_3d_f64(int degree, const PrologueArgs &a, const Tables<double> &t, cudaStream_t s);
cudaError_t launch_prologue_3d_f32(int degree, const PrologueArgs &a, const Tables<float> &t, cudaStream_t s);
cudaError_t launch_limiter_2d_f64(int degree, const LimiterArgs &a, const Tables<double> &t, cudaStream_t s);
cudaError_t launch_limiter_2d_f32(int degree, const LimiterArgs &a, const Tables<float> &t, cudaStream_t s);
cudaError_t launch_limiter_3d_f64(int degree, const LimiterArgs &a, const Tables<double> &t, cudaStream_t s);
cudaError_t launch_limiter_3d_f32(int degree, const LimiterArgs &a, const Tables<float> &t, cudaStream_t s);
// z-marching 3-D FP32-bulk stage kernel over packed total-degree storage (degrees 1 and 3)
cudaError_t launch_stage3z_packed(int degree, const StageArgs &a, const Tables<float> &t, cudaStream_t s, int *grid);
cudaError_t launch_stage_batch_2d_f64(int degree, int av, int ns, const StageArgs *descs, const int *tile_off,
                                      int nsims, int total, const Tables<double> &t, cudaStream_t s);
cudaError_t launch_stage_batch_2d_f32(int degree, int av, int ns, const StageArgs *descs, const int *tile_off,
                                      int nsims, int total, const Tables<float> &t, cudaStream_t s);
cudaError_t launch_stage_batch_3d_f64(int degree, int av, int ns, const StageArgs *descs, const int *tile_off,
                                      int nsims, int total, const Tables<double> &t, cudaStream_t s);
cudaError_t launch_stage_batch_3d_f32(int degree, int av, int ns, const StageArgs *descs, const int *tile_off,
                                      int nsims, int total, const Tables<float> &t, cudaStream_t s);
// ---- turbulence driving (Sec. 7.1), dgx_forcing.cu
constexpr int kForceModes = 16;                  // mode stride of the forcing state (3-D count)
constexpr int kForceState = 1 + 6 * kForceModes;  // last update index + (X_m, Y_m) per mode
constexpr long long kForceMaxUpdates = 100000;    // per step; more sets DG_STATUS_FORCING

// per-mode constants of the driving: physical wave vector K = 2 pi k / L and amplitude A |k|^(-5/3)
struct ForcingModes {
    int nm;
    double K[kForceModes][3];
    double amp[kForceModes];
};
// fills the modes of a dim-dimensional box of edge lengths L
void forcing_modes(int dim, const double *L, double amp, ForcingModes *fm);
// host-built per-axis tables exp(i 2 pi k x / L) at every (cell, Gauss node) along each axis,
// k = -2..2: [(cell * (n+1) + i) * 5 + k + 2] (cos, sin); returns the offsets of the axes
void forcing_phase_tables(int dim, const int *N, const double *L, int degree, double *out, long long *off);
void gauss_nodes(int q, double *x);
// advance = 1: apply the driving updates due at time *t to fstate; then (either way) write the
// projected, scaled complex amplitudes (Re s_m, Im s_m) of fstate to smodes [kForceModes][6]
cudaError_t launch_forcing_update(const ForcingModes &fm, int dim, double force_dt, double force_ts,
                                  unsigned long long seed, int advance, double *fstate, const double *t,
                                  double *smodes, int *status, cudaStream_t s);
// driving acceleration at every volume node: out [d][cell][node]
cudaError_t launch_forcing_eval_f64(int dim, int degree, const int *N, long long ncell, const double *tab,
                                    const long long *off, const double *smodes, double *out, cudaStream_t s);
cudaError_t launch_forcing_eval_f32(int dim, int degree, const int *N, long long ncell, const float *tab,
                                    const long long *off, const double *smodes, float *out, cudaStream_t s);

// stage and prologue tiles of a degree (tracer != 0: the stage tiles of the plans with a tracer)
void tiles_2d_f64(int degree, int tracer, int *stage, int *pro);
void tiles_2d_f32(int degree, int tracer, int *stage, int *pro);
void tiles_3d_f64(int degree, int tracer, int *stage, int *pro);
void tiles_3d_f32(int degree, int tracer, int *stage, int *pro);

}  // namespace dgx
