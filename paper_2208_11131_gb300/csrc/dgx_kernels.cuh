// Shared device code of the modal DG hot path (arXiv 2208.11131, Sec. 2-4) for sm_103a:
// tile geometry, pointwise physics, and the step-prologue kernel.  The fused stage kernel
// that uses them is in dgx_stage2.cuh.
//
// Formulation.  Each CTA owns a tile of cells plus the face-neighbour halo.
// The stage state is loaded once into shared memory and turned from modal
// weights into values at the (n+1)^d Gauss points by d sum-factorised 1-D
// passes (B[i][m] = Pt_m(x_i)).  Because n+1 Gauss points integrate the
// modal mass matrix exactly, every modal sum of Eq. time_stepping_final has
// an exact nodal counterpart:
//   volume:   sum_j g_j d_alpha phi_l(x_j) F_alpha(x_j)
//             = sum_m B-transforms of  r(m) = sum_i g_i Dn[i][m_alpha] F_alpha(i)
//   faces:    phi_l(+-1, x_k) = sum_m l_m(+-1) B[m][l_alpha] phi_t(x_k),
//   sources:  projection = B-transform of g_j s(x_j),
// so the kernel accumulates a nodal residual r and applies the transposed
// transform once at the end.  Interface recovery (Sec. 3.2, Eq.
// basisprojection) reduces to four 1-D functionals on the nodal lines normal
// to a face (Cm/Cp: recovered value, Dm/Dp: recovered normal derivative);
// tangential derivatives of the recovered state apply the nodal derivative
// along the face.  Both CTAs that share a tile-boundary face compute its flux
// with the same code from the same data, so the flux is bitwise identical on
// both sides and the scheme stays conservative without atomics.
#pragma once

#include <math.h>
#include <stdint.h>

#include "dgx_internal.h"

namespace dgx {

// ------------------------------------------------------------------ tile shape

template <int DIM, int N, int TX, int TY, int TZ>
struct Shape {
    static constexpr int Q = N + 1;
    static constexpr int NP = DIM == 2 ? Q * Q : Q * Q * Q;  // nodes (= modes) per cell
    static constexpr int NPF = DIM == 2 ? Q : Q * Q;         // nodes per face
    static constexpr int NC = DIM + 2;                       // conserved fields
    static constexpr int NFM = DIM + 3;                      // + alpha
    static constexpr int TC = TX * TY * TZ;
    __host__ __device__ static constexpr int T(int a) { return a == 0 ? TX : (a == 1 ? TY : TZ); }
    __host__ __device__ static constexpr int HB(int a) { return TC / T(a); }
    static constexpr int NHALO = 2 * (HB(0) + HB(1) + (DIM == 3 ? HB(2) : 0));
    static constexpr int NSLOT = TC + NHALO;
    __host__ __device__ static constexpr int HOFF(int a, int s)
    {
        return TC + (a > 0 ? 2 * HB(0) : 0) + (a > 1 ? 2 * HB(1) : 0) + s * HB(a);
    }
    __host__ __device__ static constexpr int NFA(int a) { return (T(a) + 1) * HB(a); }
    __host__ __device__ static constexpr int FOFF(int a) { return (a > 0 ? NFA(0) : 0) + (a > 1 ? NFA(1) : 0); }
    static constexpr int NFACE = NFA(0) + NFA(1) + (DIM == 3 ? NFA(2) : 0);
    __host__ __device__ static constexpr int S(int a) { return a == 0 ? 1 : (a == 1 ? Q : Q * Q); }

    // transverse tile index of a tile cell with respect to axis a
    __device__ static int trans(int a, int cx, int cy, int cz)
    {
        return a == 0 ? cy + TY * cz : (a == 1 ? cx + TX * cz : cx + TX * cy);
    }
    __device__ static void untrans(int a, int t, int *c)
    {
        if (a == 0) {
            c[1] = t % TY;
            c[2] = t / TY;
        } else if (a == 1) {
            c[0] = t % TX;
            c[2] = t / TX;
        } else {
            c[0] = t % TX;
            c[1] = t / TX;
        }
    }
    // transverse node index k of node j w.r.t. axis a (face numbering, increasing axes)
    __device__ static int ktrans(int a, int j)
    {
        if (DIM == 2) return a == 0 ? j / Q : j % Q;
        return a == 0 ? j / Q : (a == 1 ? (j % Q) + Q * (j / (Q * Q)) : j % (Q * Q));
    }
    // node index from position i along a and transverse node k
    __device__ static int knode(int a, int i, int k)
    {
        if (DIM == 2) return a == 0 ? i + Q * k : k + Q * i;
        return a == 0 ? i + Q * k : (a == 1 ? (k % Q) + Q * i + Q * Q * (k / Q) : k + Q * Q * i);
    }
};

// ------------------------------------------------------------------ pointwise physics (Sec. 2.1, 3.3, 4.1)

template <typename Real>
__device__ __forceinline__ Real clamp01(Real a)
{
    return a < Real(0) ? Real(0) : (a > Real(1) ? Real(1) : a);
}

// primitive variables; returns false for rho <= 0, p <= 0 or non-finite values
template <int DIM, typename Real>
__device__ __forceinline__ bool primitives(const Real *u, Real gamma, Real &rho, Real *v, Real &p, Real &cs)
{
    rho = u[0];
    const Real inv = Real(1) / rho;
    Real ke = Real(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        v[a] = u[1 + a] * inv;
        ke += u[1 + a] * v[a];
    }
    p = (gamma - Real(1)) * (u[DIM + 1] - Real(0.5) * ke);
    const bool ok = (rho > Real(0)) && (p > Real(0));
    cs = ok ? sqrt(gamma * p * inv) : Real(0);
    return ok;
}

// Euler flux along axis a (a may be a run-time value: selected by value, no run-time indexing);
// TR: a passive tracer rho c follows the energy, with flux c rho v_a (Sec. 3.4)
template <int DIM, bool TR = false, typename Real>
__device__ __forceinline__ void euler_flux(const Real *u, const Real *v, Real p, int a, Real *F)
{
    Real va = v[0], ma = u[1];
#pragma unroll
    for (int b = 1; b < DIM; ++b) {
        va = b == a ? v[b] : va;
        ma = b == a ? u[1 + b] : ma;
    }
    F[0] = ma;
#pragma unroll
    for (int b = 0; b < DIM; ++b) F[1 + b] = u[1 + b] * va + (b == a ? p : Real(0));
    F[DIM + 1] = (u[DIM + 1] + p) * va;
    if constexpr (TR) F[DIM + 2] = u[DIM + 2] * va;
}

// HLLC with Davis wave speeds (Toro); passive transverse momentum and (TR) a passive tracer carried
// in the star state with its side's concentration.  Returns false on a bad state.
// Written without pointers to local arrays and without early returns: the side values that enter
// the star state are chosen by value selects, so every array stays in registers.
template <int DIM, bool TR = false, typename Real>
__device__ __forceinline__ bool hllc(const Real *uL, const Real *uR, Real gamma, int a, Real *F, Real &cL, Real &cR)
{
    constexpr int NC = DIM + 2 + (TR ? 1 : 0);
    Real rL, rR, pL, pR, vL[3], vR[3];
    bool ok = primitives<DIM>(uL, gamma, rL, vL, pL, cL);
    ok = primitives<DIM>(uR, gamma, rR, vR, pR, cR) && ok;
    Real vnL = vL[0], vnR = vR[0];
#pragma unroll
    for (int b = 1; b < DIM; ++b) {
        vnL = b == a ? vL[b] : vnL;
        vnR = b == a ? vR[b] : vnR;
    }
    const Real SL = fmin(vnL - cL, vnR - cR);
    const Real SR = fmax(vnL + cL, vnR + cR);
    const Real num = pR - pL + rL * vnL * (SL - vnL) - rR * vnR * (SR - vnR);
    const Real den = rL * (SL - vnL) - rR * (SR - vnR);
    const Real Ss = num / den;
    // region: 0 = left state, 1 = left star, 2 = right star, 3 = right state
    const int region = SL >= Real(0) ? 0 : (Ss >= Real(0) ? 1 : (SR >= Real(0) ? 2 : 3));
    const bool left = region <= 1;
    Real uK[NC], vK[DIM];
#pragma unroll
    for (int f = 0; f < NC; ++f) uK[f] = left ? uL[f] : uR[f];
#pragma unroll
    for (int b = 0; b < DIM; ++b) vK[b] = left ? vL[b] : vR[b];
    const Real rK = left ? rL : rR, pK = left ? pL : pR, vnK = left ? vnL : vnR;
    const Real SK = left ? SL : SR;
    // physical flux of the chosen side
    Real mK = uK[1];
#pragma unroll
    for (int b = 1; b < DIM; ++b) mK = b == a ? uK[1 + b] : mK;
    F[0] = mK;
#pragma unroll
    for (int b = 0; b < DIM; ++b) F[1 + b] = uK[1 + b] * vnK + (b == a ? pK : Real(0));
    F[DIM + 1] = (uK[DIM + 1] + pK) * vnK;
    if constexpr (TR) F[DIM + 2] = uK[DIM + 2] * vnK;
    if (region == 1 || region == 2) {
        const Real fac = rK * (SK - vnK) / (SK - Ss);
        Real us[NC];
        us[0] = fac;
#pragma unroll
        for (int b = 0; b < DIM; ++b) us[1 + b] = fac * (b == a ? Ss : vK[b]);
        us[DIM + 1] = fac * (uK[DIM + 1] / rK + (Ss - vnK) * (Ss + pK / (rK * (SK - vnK))));
        if constexpr (TR) us[DIM + 2] = fac * (uK[DIM + 2] / rK);
#pragma unroll
        for (int f = 0; f < NC; ++f) F[f] += SK * (us[f] - uK[f]);
    }
    return ok;
}

template <int DIM, bool TR = false, typename Real>
__device__ __forceinline__ bool hllc(const Real *uL, const Real *uR, Real gamma, int a, Real *F)
{
    Real cL, cR;
    return hllc<DIM, TR>(uL, uR, gamma, a, F, cL, cR);
}

// Navier-Stokes flux along axis a (Sec. 3.3): (0, Pi_a, v.Pi_a + kappa (gamma-1) rho d_a u_int),
// Pi = nu rho (grad v + grad v^T - 2/3 div v I); TR: the tracer row eta rho d_a c =
// eta (d_a (rho c) - c d_a rho) (Sec. 3.4).  grad[b][f] is the physical gradient.
template <int DIM, bool TR = false, typename Real>
__device__ __forceinline__ void ns_flux(const Real *u, const Real (*grad)[DIM + 2 + (TR ? 1 : 0)], Real gamma,
                                        Real nu, Real kappa, Real eta, int a, Real *F)
{
    const Real rho = u[0];
    const Real inv = Real(1) / rho;
    Real v[DIM], dv[DIM][DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) v[b] = u[1 + b] * inv;
    Real div = Real(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) dv[b][c] = (grad[b][1 + c] - v[c] * grad[b][0]) * inv;
        div += dv[b][b];
    }
    const Real nr = nu * rho;
    Real work = Real(0);
    F[0] = Real(0);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        Real pi = nr * (dv[a][c] + dv[c][a] - (c == a ? Real(2.0 / 3.0) * div : Real(0)));
        F[1 + c] = pi;
        work += v[c] * pi;
    }
    Real duint = (grad[a][DIM + 1] - u[DIM + 1] * inv * grad[a][0]) * inv;
#pragma unroll
    for (int c = 0; c < DIM; ++c) duint -= v[c] * dv[a][c];
    F[DIM + 1] = work + kappa * (gamma - Real(1)) * rho * duint;
    if constexpr (TR) F[DIM + 2] = eta * (grad[a][DIM + 2] - u[DIM + 2] * inv * grad[a][0]);
}

// Navier-Stokes fluxes along all DIM axes at one point (the rows of ns_flux for a = 0..DIM-1),
// with the velocity gradient and its divergence formed once: F[a][f]
template <int DIM, typename Real>
__device__ __forceinline__ void ns_flux_all(const Real *u, const Real (*grad)[DIM + 2], Real gamma, Real nu,
                                            Real kappa, Real (*F)[DIM + 2])
{
    const Real rho = u[0];
    const Real inv = Real(1) / rho;
    Real v[DIM], dv[DIM][DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) v[b] = u[1 + b] * inv;
    Real div = Real(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) dv[b][c] = (grad[b][1 + c] - v[c] * grad[b][0]) * inv;
        div += dv[b][b];
    }
    const Real nr = nu * rho;
    const Real eint = u[DIM + 1] * inv;
    const Real kg = kappa * (gamma - Real(1)) * rho;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        Real work = Real(0);
        F[a][0] = Real(0);
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            Real pi = nr * (dv[a][c] + dv[c][a] - (c == a ? Real(2.0 / 3.0) * div : Real(0)));
            F[a][1 + c] = pi;
            work += v[c] * pi;
        }
        Real duint = (grad[a][DIM + 1] - eint * grad[a][0]) * inv;
#pragma unroll
        for (int c = 0; c < DIM; ++c) duint -= v[c] * dv[a][c];
        F[a][DIM + 1] = work + kg * duint;
    }
}

// ------------------------------------------------------------------ shared memory plan

template <int DIM, int N, typename Real, int TX, int TY, int TZ>
struct ProloguePlan {
    using S = Shape<DIM, N, TX, TY, TZ>;
    static constexpr int Q = S::Q;
    static constexpr int TAB = (Q * Q + 3) / 4 * 4;
    static constexpr int SZ = S::NC * S::TC * S::NP;
    static constexpr int NREAL = TAB + 2 * SZ;
    static constexpr size_t BYTES = sizeof(Real) * (size_t)NREAL + sizeof(int) * (size_t)S::TC;
};

template <typename Real>
__device__ __forceinline__ Real ld_cg(const Real *p)
{
    return *p;
}

// global cell index of a tile slot (tile cell or face-neighbour halo), -1 if none
template <class S>
__device__ __forceinline__ int slot_global(int slot, const int *o, const int *V, const int *N, const int *bc)
{
    constexpr int TX = S::T(0), TY = S::T(1);
    int c[3];
    if (slot < S::TC) {
        c[0] = slot % TX;
        c[1] = (slot / TX) % TY;
        c[2] = slot / (TX * TY);
        if (c[0] >= V[0] || c[1] >= V[1] || c[2] >= V[2]) return -1;
        return (o[0] + c[0]) + N[0] * ((o[1] + c[1]) + N[1] * (o[2] + c[2]));
    }
    int r = slot - S::TC;
    int a = 0;
    for (; a < 3; ++a) {
        if (r < 2 * S::HB(a)) break;
        r -= 2 * S::HB(a);
    }
    const int s = r / S::HB(a);
    const int t = r % S::HB(a);
    c[0] = c[1] = c[2] = 0;
    S::untrans(a, t, c);
    int g[3];
    for (int b = 0; b < 3; ++b) {
        if (b == a) continue;
        if (c[b] >= V[b]) return -1;
        g[b] = o[b] + c[b];
    }
    int ca = s == 0 ? o[a] - 1 : o[a] + V[a];
    if (ca < 0 || ca >= N[a]) {
        if (bc[a] != 0) return -1;
        ca = (ca + N[a]) % N[a];
    }
    g[a] = ca;
    return g[0] + N[0] * (g[1] + N[1] * g[2]);
}

// ------------------------------------------------------------------ step prologue: sensor + CFL speeds

template <int DIM, int N, typename Real, int TX, int TY, int TZ>
__global__ void __launch_bounds__(256) prologue_kernel(const PrologueArgs A, const Tables<Real> Tg)
{
    using S = Shape<DIM, N, TX, TY, TZ>;
    using PL = ProloguePlan<DIM, N, Real, TX, TY, TZ>;
    constexpr int Q = S::Q, NP = S::NP, NC = S::NC, TC = S::TC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *sm = reinterpret_cast<Real *>(smem_raw);
    Real *tB = sm;
    Real *sU = sm + PL::TAB, *sW = sU + PL::SZ;
    int *sG = reinterpret_cast<int *>(sm + PL::NREAL);
    __shared__ double red[2][32];
    __shared__ int s_bad;

    const int tid = threadIdx.x, nth = blockDim.x;
    int b = blockIdx.x;
    const int tx = b % A.ntile[0];
    b /= A.ntile[0];
    const int ty = b % A.ntile[1];
    const int tz = b / A.ntile[1];
    const int o[3] = {tx * TX, ty * TY, tz * TZ};
    const int V[3] = {min(TX, A.N[0] - o[0]), min(TY, A.N[1] - o[1]), DIM == 3 ? min(TZ, A.N[2] - o[2]) : 1};
    for (int i = tid; i < Q * Q; i += nth) tB[i] = Tg.B[i / Q][i % Q];
    for (int c = tid; c < TC; c += nth) {
        const int cc[3] = {c % TX, (c / TX) % TY, c / (TX * TY)};
        sG[c] = (cc[0] < V[0] && cc[1] < V[1] && cc[2] < V[2])
                    ? (o[0] + cc[0]) + A.N[0] * ((o[1] + cc[1]) + A.N[1] * (o[2] + cc[2]))
                    : -1;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const Real *u = static_cast<const Real *>(A.u);
    {
        // the tile's modes, up to 32 loads of a thread in flight at once (the block has 256 threads)
        constexpr int NL = NC * TC * NP, NTH = 256, PER = (NL + NTH - 1) / NTH, CH = PER < 32 ? PER : 32;
        const int ms = A.cmap ? A.ms : NP;
        for (int j0 = 0; j0 < PER; j0 += CH) {
            Real v[CH];
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) {
                const int idx = tid + NTH * (j0 + jj);
                v[jj] = Real(0);
                if (idx < NL) {
                    const int l = idx % NP, fc = idx / NP;
                    const int c = fc % TC, f = fc / TC;
                    const int g = sG[c];
                    // packed total-degree storage: the modes outside the basis are not stored (zero)
                    const int sl = A.cmap ? A.cmap[l] : l;
                    if (g >= 0 && sl >= 0) v[jj] = u[((size_t)f * A.ncell + g) * ms + sl];
                }
            }
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) {
                const int idx = tid + NTH * (j0 + jj);
                if (idx < NL) sU[idx] = v[jj];
            }
        }
    }
    __syncthreads();
    if (A.update_sensor) {
        const double dt_prev = A.dtp[0];
        const double step = A.dtp[1];
        // TPC threads per cell (a power of two dividing 32) sum strided modes, then combine by shuffles
        constexpr int TPC0 = 256 / TC < 1 ? 1 : 256 / TC;
        constexpr int TPC = TPC0 >= 32 ? 32 : TPC0 >= 16 ? 16 : TPC0 >= 8 ? 8 : TPC0 >= 4 ? 4 : TPC0 >= 2 ? 2 : 1;
        constexpr int CPR = 256 / TPC;  // cells per round of the block
        for (int c0 = 0; c0 < TC; c0 += CPR) {
            const int c = c0 + tid / TPC, sub = tid % TPC;
            const int g = c < TC ? sG[c] : -1;
            Real hi = Real(0), all = Real(0);
            if (g >= 0) {
                for (int l = sub; l < NP; l += TPC) {
                    const Real w = sU[c * NP + l];  // density field (f = 0)
                    const int l0 = l % Q, l1 = (l / Q) % Q, l2 = DIM == 3 ? l / (Q * Q) : 0;
                    // the modes the degree-(n-1) basis lacks (Sec. 4.1)
                    const bool top = N > 0 && (A.total_degree ? (l0 + l1 + l2 == N)
                                                              : (l0 == N || l1 == N || (DIM == 3 && l2 == N)));
                    all += w * w;
                    if (top) hi += w * w;
                }
            }
#pragma unroll
            for (int off = TPC / 2; off > 0; off >>= 1) {
                all += __shfl_xor_sync(0xffffffffu, all, off);
                hi += __shfl_xor_sync(0xffffffffu, hi, off);
            }
            if (g < 0 || sub != 0) continue;
            const double Sk = all > Real(0) ? (double)(hi / all) : 0.0;
            double dlog = 0.0;
            // S is floored four decades below the onset threshold: below that its value is rounding
            // noise of the higher modes, and a log of noise would turn into a source of size noise / dt
            const double s_floor = 1e-4 * A.s_on;
            if (step > 0.0 && dt_prev > 0.0) {
                if constexpr (sizeof(Real) == 4) {  // FP32 sensor: its logarithm in FP32 as well
                    const float sf = (float)s_floor;
                    dlog = (double)((logf(fmaxf((float)Sk, sf)) - logf(fmaxf((float)A.S_prev[g], sf))) /
                                    (float)dt_prev);
                } else {
                    dlog = (log(fmax(Sk, s_floor)) - log(fmax(A.S_prev[g], s_floor))) / dt_prev;
                }
            }
            A.wig[g] = (Sk > A.s_on) ? A.f_w * fmax(0.0, dlog) : 0.0;
            A.S_prev[g] = Sk;
        }
    }
    // modal -> nodal for the conserved fields
    Real *src = sU, *dst = sW;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const int Sa = S::S(a);
        for (int idx = tid; idx < NC * TC * NP; idx += nth) {
            const int j = idx % NP, fc = idx / NP;
            if (sG[fc % TC] < 0) continue;
            const int i = (j / Sa) % Q;
            const Real *p = src + fc * NP + (j - i * Sa);
            Real acc = Real(0);
#pragma unroll
            for (int m = 0; m < Q; ++m) acc = fma(tB[i * Q + m], p[m * Sa], acc);
            dst[idx] = acc;
        }
        Real *t = src;
        src = dst;
        dst = t;
        __syncthreads();
    }
    double cmax = 0.0, vmax = 0.0;
    int bad = 0;
    const Real gamma = (Real)A.gamma;
    for (int idx = tid; idx < TC * NP; idx += nth) {
        const int c = idx / NP, j = idx % NP;
        if (sG[c] < 0) continue;
        Real uu[NC];
#pragma unroll
        for (int f = 0; f < NC; ++f) uu[f] = src[(f * TC + c) * NP + j];
        Real rho, v[3], p, cs;
        if (!primitives<DIM>(uu, gamma, rho, v, p, cs)) bad = 1;
        Real v2 = Real(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) v2 += v[a] * v[a];
        cmax = fmax(cmax, (double)cs);
        vmax = fmax(vmax, (double)sqrt(v2));
    }
    // block max-reduction: warp shuffle, then one value per warp
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, off));
        vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    }
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        red[0][warp] = cmax;
        red[1][warp] = vmax;
    }
    if (bad) s_bad = 1;
    __syncthreads();
    if (tid == 0) {
        double c0 = 0.0, v0 = 0.0;
        for (int w = 0; w < (nth + 31) / 32; ++w) {
            c0 = fmax(c0, red[0][w]);
            v0 = fmax(v0, red[1][w]);
        }
        A.partial[2 * blockIdx.x + 0] = c0;
        A.partial[2 * blockIdx.x + 1] = v0;
        if (s_bad) atomicOr(A.status, DG_STATUS_NONPHYS);
    }
}

// ------------------------------------------------------------------ launchers

template <int DIM, int N, typename Real, int TX, int TY, int TZ>
cudaError_t run_prologue(const PrologueArgs &a, const Tables<Real> &t, cudaStream_t s)
{
    using PL = ProloguePlan<DIM, N, Real, TX, TY, TZ>;
    auto k = prologue_kernel<DIM, N, Real, TX, TY, TZ>;
    static_assert(PL::BYTES <= 227 * 1024, "prologue tile exceeds shared memory");
    static KernelSetup ks;
    cudaError_t e = kernel_setup(ks, k, 256, PL::BYTES);
    if (e != cudaSuccess) return e;
    const int blocks = a.ntile[0] * a.ntile[1] * a.ntile[2];
    if (blocks == 0) return cudaSuccess;
    k<<<blocks, 256, PL::BYTES, s>>>(a, t);
    return cudaGetLastError();
}

}  // namespace dgx
