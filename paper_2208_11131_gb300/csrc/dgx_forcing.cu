// Turbulence driving of Sec. 7.1 ("Driving"): a solenoidal acceleration field made of Fourier
// modes 2pi/L <= |k| <= 2 (2pi/L) with amplitude A |k|^(-5/3), whose complex vector
// coefficients follow Ornstein-Uhlenbeck processes updated at times j * force_dt.
//
// GPU organisation:
//  * forcing_update_kernel (one block, one thread per (mode, component)): applies every update
//    due at the step's start time t (read from device memory, so a step stays free of host
//    synchronisation and can be graph-captured), then projects each mode onto the plane normal
//    to its wave vector and scales it;
//  * forcing_eval_kernel: the acceleration at every volume Gauss node, from per-axis phase
//    tables exp(i K_a x_a) built once on the host (no transcendental functions on the device)
//    and the mode list fixed at compile time, written to [d][cell][node] for the stage kernel.
//
// Exact OU update over an interval: X <- f X + sqrt(1 - f^2) xi, f = exp(-force_dt / t_s),
// unit stationary variance; update 0 draws the stationary state.  Normal draws xi: Box-Muller
// (1958) on two outputs of the SplitMix64 generator (Steele, Lea & Flood 2014) used
// counter-based (output i of seed s = mix(s + (i+1) * golden gamma)); the counter of update j,
// mode m, component q (0..2 real, 3..5 imaginary part) is (16 j + m) * 6 + q.
#include <math.h>

#include "dgx_internal.h"

namespace dgx {

namespace {

// integer wave vectors of the driving, 1 <= |k|^2 <= 4, first non-zero component positive,
// ordered kz (outer), ky, kx (inner)
template <int DIM>
struct ModeList {
    int n;
    int k[kForceModes][3];
};

template <int DIM>
__host__ __device__ constexpr ModeList<DIM> mode_list()
{
    ModeList<DIM> L{};
    L.n = 0;
    const int zr = DIM == 3 ? 2 : 0;
    for (int kz = -zr; kz <= zr; ++kz)
        for (int ky = -2; ky <= 2; ++ky)
            for (int kx = -2; kx <= 2; ++kx) {
                const int k2 = kx * kx + ky * ky + kz * kz;
                if (k2 < 1 || k2 > 4) continue;
                const int first = kx != 0 ? kx : (ky != 0 ? ky : kz);
                if (first < 0) continue;
                L.k[L.n][0] = kx;
                L.k[L.n][1] = ky;
                L.k[L.n][2] = kz;
                ++L.n;
            }
    return L;
}

__device__ __forceinline__ unsigned long long splitmix(unsigned long long seed, unsigned long long i)
{
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double unit_open(unsigned long long seed, unsigned long long i)
{
    return ((double)(splitmix(seed, i) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ double normal_draw(unsigned long long seed, unsigned long long c)
{
    const double u1 = unit_open(seed, 2ull * c), u2 = unit_open(seed, 2ull * c + 1ull);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

// advance = 0: only the projection of the current state (no update, no initial draw)
__global__ void forcing_update_kernel(const ForcingModes fm, int dim, double decay, double noise, double force_dt,
                                      unsigned long long seed, int advance, double *fstate, const double *t_ptr,
                                      double *smodes, int *status)
{
    __shared__ double sx[6 * kForceModes];
    const int tid = threadIdx.x;  // 6 m + q
    const double t = *t_ptr;
    const double j0 = fstate[0];
    const bool active = tid < 6 * fm.nm && (tid % 3) < dim;
    long long j = (long long)j0;
    double x = active ? fstate[1 + tid] : 0.0;
    bool over = false;
    if (advance) {
        if (j0 < 0.0) {
            j = 0;
            if (active) x = normal_draw(seed, (unsigned long long)tid);
        }
        long long count = 0;
        // every thread sees the same t and j: the trip count is uniform
        while ((double)(j + 1) * force_dt <= t) {
            if (++count > kForceMaxUpdates) {
                over = true;
                break;
            }
            ++j;
            if (active) x = decay * x + noise * normal_draw(seed, (unsigned long long)j * (6 * kForceModes) + tid);
        }
    }
    if (tid < 6 * kForceModes) sx[tid] = x;
    __syncthreads();
    if (advance) {
        if (active) fstate[1 + tid] = x;
        if (tid == 0) {
            fstate[0] = (double)j;
            if (over) atomicOr(status, DG_STATUS_FORCING);
        }
    }
    if (tid < fm.nm) {
        const double *X = sx + 6 * tid, *Y = X + 3;
        double KX = 0.0, KY = 0.0, K2 = 0.0;
        for (int a = 0; a < dim; ++a) {
            KX += fm.K[tid][a] * X[a];
            KY += fm.K[tid][a] * Y[a];
            K2 += fm.K[tid][a] * fm.K[tid][a];
        }
        for (int a = 0; a < 3; ++a) {
            const bool in = a < dim;
            smodes[6 * tid + a] = in ? fm.amp[tid] * (X[a] - fm.K[tid][a] * KX / K2) : 0.0;
            smodes[6 * tid + 3 + a] = in ? fm.amp[tid] * (Y[a] - fm.K[tid][a] * KY / K2) : 0.0;
        }
    }
}

// one thread per x-line of Q volume nodes (fixed y and z node of a cell): the y/z phase products of
// every mode are formed once per line and multiplied by each node's x phase.  Q is a compile-time
// constant, so the splits of the flat index are multiplications, and the cell split uses 32-bit
// arithmetic (cells < 2^31)
template <int DIM, int Q, typename Real>
__global__ void __launch_bounds__(256) forcing_eval_kernel(int N0, int N1, long long ncell, const Real *tab,
                                                           long long off1, long long off2, const double *smodes,
                                                           Real *out)
{
    constexpr ModeList<DIM> ML = mode_list<DIM>();
    constexpr int NP = DIM == 2 ? Q * Q : Q * Q * Q;
    constexpr int NL = NP / Q;  // x-lines per cell
    __shared__ Real sm[6 * kForceModes];
    for (int i = threadIdx.x; i < 6 * kForceModes; i += blockDim.x) sm[i] = (Real)smodes[i];
    __syncthreads();
    const long long total = ncell * NL;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(idx / NL);
        const int line = (int)(idx - (long long)cell * NL);
        const int c01 = cell / N0;
        const int c0 = cell - c01 * N0;
        const int c2 = c01 / N1;
        const int c1 = c01 - c2 * N1;
        const int j1 = line % Q, j2 = line / Q;
        // exp(i K_a x_a) for k_a = -2..2 at this line's y and z nodes
        Real er1[5], ei1[5], er2[5], ei2[5];
        const Real *t1 = tab + off1 + (c1 * Q + j1) * 10;
        const Real *t2 = tab + off2 + (c2 * Q + j2) * 10;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            er1[k] = t1[2 * k];
            ei1[k] = t1[2 * k + 1];
            er2[k] = DIM == 3 ? t2[2 * k] : Real(1);
            ei2[k] = DIM == 3 ? t2[2 * k + 1] : Real(0);
        }
        // y/z part of every mode's phase
        Real pr[ML.n], pi[ML.n];
#pragma unroll
        for (int m = 0; m < ML.n; ++m) {
            const int ky = ML.k[m][1] + 2, kz = ML.k[m][2] + 2;
            pr[m] = er1[ky] * er2[kz] - ei1[ky] * ei2[kz];
            pi[m] = er1[ky] * ei2[kz] + ei1[ky] * er2[kz];
        }
        Real *o0 = out + (long long)cell * NP + (long long)line * Q;
        // one x node at a time (the amplitudes are re-read from shared memory per node rather than
        // held in registers for the whole line)
#pragma unroll 1
        for (int x = 0; x < Q; ++x) {
            const Real *t0 = tab + (c0 * Q + x) * 10;
            Real er0[5], ei0[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                er0[k] = t0[2 * k];
                ei0[k] = t0[2 * k + 1];
            }
            Real s[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
            for (int m = 0; m < ML.n; ++m) {
                const int kx = ML.k[m][0] + 2;
                const Real re = er0[kx] * pr[m] - ei0[kx] * pi[m];
                const Real im = er0[kx] * pi[m] + ei0[kx] * pr[m];
#pragma unroll
                for (int a = 0; a < DIM; ++a) s[a] += sm[6 * m + a] * re - sm[6 * m + 3 + a] * im;
            }
#pragma unroll
            for (int a = 0; a < DIM; ++a) o0[(long long)a * ncell * NP + x] = s[a];
        }
    }
}

template <int DIM, int Q, typename Real>
cudaError_t launch_eval(const int *N, long long ncell, const Real *tab, const long long *off, const double *smodes,
                        Real *out, cudaStream_t s)
{
    constexpr int NP = DIM == 2 ? Q * Q : Q * Q * Q;
    const long long total = ncell * (NP / Q);
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) return cudaSuccess;
    forcing_eval_kernel<DIM, Q, Real><<<(unsigned)blocks, 256, 0, s>>>(N[0], N[1], ncell, tab, off[1],
                                                                        DIM == 3 ? off[2] : 0, smodes, out);
    return cudaGetLastError();
}

template <int DIM, typename Real>
cudaError_t launch_eval_dim(int degree, const int *N, long long ncell, const Real *tab, const long long *off,
                            const double *smodes, Real *out, cudaStream_t s)
{
    switch (degree) {
    case 0: return launch_eval<DIM, 1, Real>(N, ncell, tab, off, smodes, out, s);
    case 1: return launch_eval<DIM, 2, Real>(N, ncell, tab, off, smodes, out, s);
    case 2: return launch_eval<DIM, 3, Real>(N, ncell, tab, off, smodes, out, s);
    case 3: return launch_eval<DIM, 4, Real>(N, ncell, tab, off, smodes, out, s);
    case 4: return launch_eval<DIM, 5, Real>(N, ncell, tab, off, smodes, out, s);
    case 5: return launch_eval<DIM, 6, Real>(N, ncell, tab, off, smodes, out, s);
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t run_forcing_eval(int dim, int degree, const int *N, long long ncell, const Real *tab, const long long *off,
                             const double *smodes, Real *out, cudaStream_t s)
{
    if (dim == 2) return launch_eval_dim<2, Real>(degree, N, ncell, tab, off, smodes, out, s);
    return launch_eval_dim<3, Real>(degree, N, ncell, tab, off, smodes, out, s);
}

}  // namespace

void forcing_modes(int dim, const double *L, double amp, ForcingModes *fm)
{
    const double two_pi = 6.283185307179586476925286766559;
    ForcingModes F{};
    auto fill = [&](const auto &ML) {
        F.nm = ML.n;
        for (int m = 0; m < ML.n; ++m) {
            double kk = 0.0;
            for (int a = 0; a < 3; ++a) {
                F.K[m][a] = a < dim ? two_pi * ML.k[m][a] / L[a] : 0.0;
                kk += (double)ML.k[m][a] * ML.k[m][a];
            }
            F.amp[m] = amp * pow(sqrt(kk), -5.0 / 3.0);
        }
    };
    if (dim == 2) fill(mode_list<2>());
    else fill(mode_list<3>());
    *fm = F;
}

void forcing_phase_tables(int dim, const int *N, const double *L, int degree, double *out, long long *off)
{
    const int Q = degree + 1;
    double xg[kMaxQ];
    gauss_nodes(Q, xg);
    const long double two_pi = 6.283185307179586476925286766559L;
    long long o = 0;
    for (int a = 0; a < 3; ++a) {
        off[a] = o;
        if (a >= dim) continue;
        const long double h = (long double)L[a] / N[a];
        for (int c = 0; c < N[a]; ++c)
            for (int i = 0; i < Q; ++i) {
                const long double x = (c + 0.5L + 0.5L * xg[i]) * h;  // from the box's lower corner
                for (int k = -2; k <= 2; ++k) {
                    const long double th = two_pi * k * x / L[a];
                    out[o + ((long long)c * Q + i) * 10 + 2 * (k + 2)] = (double)cosl(th);
                    out[o + ((long long)c * Q + i) * 10 + 2 * (k + 2) + 1] = (double)sinl(th);
                }
            }
        o += (long long)N[a] * Q * 10;
    }
}

cudaError_t launch_forcing_update(const ForcingModes &fm, int dim, double force_dt, double force_ts,
                                  unsigned long long seed, int advance, double *fstate, const double *t,
                                  double *smodes, int *status, cudaStream_t s)
{
    const double f = exp(-force_dt / force_ts);
    forcing_update_kernel<<<1, 6 * kForceModes, 0, s>>>(fm, dim, f, sqrt(1.0 - f * f), force_dt, seed, advance,
                                                        fstate, t, smodes, status);
    return cudaGetLastError();
}

cudaError_t launch_forcing_eval_f64(int dim, int degree, const int *N, long long ncell, const double *tab,
                                    const long long *off, const double *smodes, double *out, cudaStream_t s)
{
    return run_forcing_eval<double>(dim, degree, N, ncell, tab, off, smodes, out, s);
}

cudaError_t launch_forcing_eval_f32(int dim, int degree, const int *N, long long ncell, const float *tab,
                                    const long long *off, const double *smodes, float *out, cudaStream_t s)
{
    return run_forcing_eval<float>(dim, degree, N, ncell, tab, off, smodes, out, s);
}

}  // namespace dgx
