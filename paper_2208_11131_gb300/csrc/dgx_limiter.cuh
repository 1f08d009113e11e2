// Positivity limiter of Sec. 4.2, applied to a Runge-Kutta stage state, one warp per cell.
//
// For every cell: rho_bottom = 1e-6 mean(rho) and p_bottom = 1e-6 p(mean state).  The state is
// evaluated at the volume Gauss points and at the Gauss points of the 2d faces -- all of them
// points of the tensor grid {x_1..x_Q, -1, +1}^d with at most one coordinate at +-1 -- by d
// sum-factorised passes that widen one axis at a time from Q to Q+2 values.  If the minimum
// density is below rho_bottom, the higher modes of every conserved field are scaled by
// theta = (mean - rho_bottom) / (mean - rho_min).  Then the higher modes are halved until the
// minimum pressure is at least p_bottom, at most 60 times.  Along u(s) = mean + s (u - mean)
// the pressure is concave in s and above p_bottom at s = 0, so each point needs all halvings
// up to its own first admissible one; the cell takes the largest count.  The total factor
// theta 2^-k is applied in one multiplication (halving is exact, so this is the same as
// scaling by theta and halving k times).
#pragma once

#include <type_traits>

#include "dgx_kernels.cuh"

namespace dgx {


template <int DIM, int N, typename Real, bool TR>
struct LimiterPlan {
    static constexpr int Q = N + 1;
    static constexpr int E = Q + 2;  // Gauss points, then -1, then +1
    static constexpr int NP = DIM == 2 ? Q * Q : Q * Q * Q;
    static constexpr int NE = DIM == 2 ? E * E : E * E * E;
    static constexpr int NC = DIM + 2 + (TR ? 1 : 0);  // conserved fields (with a passive tracer)
    static constexpr size_t PER_CELL = sizeof(Real) * (size_t)NC * (NP + 2 * NE);
    static constexpr int CPB_RAW = (int)((96 * 1024) / PER_CELL);
    static constexpr int CPB = CPB_RAW >= 8 ? 8 : (CPB_RAW < 1 ? 1 : CPB_RAW);  // cells (= warps) per CTA
    static constexpr size_t BYTES = sizeof(Real) * (size_t)(E * Q) + PER_CELL * CPB;
};

// LAST: the state is the FP64 u^{n+1} (A.last), else u_base + delta in Real
template <int DIM, int N, typename Real, bool TR, bool LAST>
__global__ void limiter_kernel(const LimiterArgs A, const Tables<Real> Tg)
{
    using PL = LimiterPlan<DIM, N, Real, TR>;
    constexpr int Q = PL::Q, E = PL::E, NP = PL::NP, NE = PL::NE, NC = PL::NC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *tE = reinterpret_cast<Real *>(smem_raw);  // [E][Q]: Pt_m at x_i, then at -1, +1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Real *sM = tE + E * Q + (size_t)warp * NC * (NP + 2 * NE);
    Real *sA = sM + NC * NP;
    Real *sB = sA + NC * NE;

    for (int i = threadIdx.x; i < E * Q; i += blockDim.x) {
        const int r = i / Q, m = i % Q;
        if (r < Q) {
            tE[i] = Tg.B[r][m];
        } else {
            // Pt_m(-1) = (-1)^m sqrt(2m+1), Pt_m(+1) = sqrt(2m+1)
            const Real s = sqrt(Real(2 * m + 1));
            tE[i] = (r == Q && (m & 1)) ? -s : s;
        }
    }
    __syncthreads();

    const Real *ub = static_cast<const Real *>(A.ubase);
    Real *dl = static_cast<Real *>(A.delta);
    // packed total-degree storage: cmap gives the stored index of a tensor mode (-1: not stored, zero)
    const int ms = A.cmap ? A.ms : NP;
    // persistent: each warp takes cells in turn, so a cell that needs the full evaluation holds only
    // its own warp (and that warp's shared memory), not a whole CTA.  The loads of a warp's next cell
    // are issued before the current cell is tested, so they are in flight while it is.
    // The cell's modes [field][mode]: element i = lane + 32 j in register j of the lane.
    constexpr int NI = NC * NP, NJ = (NI + 31) / 32;
    using Raw = typename std::conditional<LAST, double, Real>::type;
    Raw ra[NJ], rb[NJ];  // raw loads of the next cell: u^{n+1}, or u_base and delta
    auto fetch = [&](long long c) {
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int i = lane + 32 * j;
            ra[j] = Raw(0);
            rb[j] = Raw(0);
            if (i < NI && c < A.ncell) {
                const int f = i / NP, l = i % NP;
                const int sl = A.cmap ? A.cmap[l] : l;
                if (sl >= 0) {
                    const size_t gi = ((size_t)f * A.ncell + c) * ms + sl;
                    if constexpr (LAST) {
                        ra[j] = A.ufull[gi];
                    } else {
                        ra[j] = ub[gi];
                        rb[j] = dl[gi];
                    }
                }
            }
        }
    };
    // prefetching where the raw registers stay within 40 per thread (the high-degree FP64 plans
    // load each cell when they reach it)
    constexpr bool PF = NJ * sizeof(Raw) * (LAST ? 1 : 2) <= 160;
    const long long stride = (long long)gridDim.x * PL::CPB;
    if constexpr (PF) fetch((long long)blockIdx.x * PL::CPB + warp);
    for (long long cell = (long long)blockIdx.x * PL::CPB + warp; cell < A.ncell; cell += stride) {
        __syncwarp();  // the last cell's write-back has read its shared memory
        if constexpr (!PF) fetch(cell);
        Real w[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) w[j] = LAST ? (Real)ra[j] : Real(ra[j] + rb[j]);
        if constexpr (PF) fetch(cell + stride);

        // A test from the modes alone.  On the reference cell |phi_l| <= c_l = prod_a sqrt(2 l_a + 1), so
        // every point value of field f lies within w_0 +- V_f, V_f = sum_{l>0} c_l |w_l|.  If the density
        // and pressure lower bounds of those intervals clear rho_bottom and p_bottom by a margin far above
        // the rounding of the point evaluation, the evaluation below would find theta = 1 and no halving
        // at every point -- the case in which it leaves the cell as it is -- so the cell is left now.
        {
            const Real gam = (Real)A.gamma;
            Real var[NC];
#pragma unroll
            for (int f = 0; f < NC; ++f) var[f] = Real(0);
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int i = lane + 32 * j;
                const int fi = i / NP, l = i % NP;
                const int l0 = l % Q, l1 = (l / Q) % Q, l2 = DIM == 3 ? l / (Q * Q) : 0;
                const Real c = (i < NI && l > 0) ? sqrt(Real((2 * l0 + 1) * (2 * l1 + 1) * (2 * l2 + 1))) : Real(0);
                const Real t = c * fabs(w[j]);
#pragma unroll
                for (int f = 0; f < NC; ++f) var[f] += fi == f ? t : Real(0);
            }
#pragma unroll
            for (int f = 0; f < NC; ++f)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) var[f] += __shfl_xor_sync(0xffffffffu, var[f], off);
            Real m[NC];
#pragma unroll
            for (int f = 0; f < NC; ++f) m[f] = __shfl_sync(0xffffffffu, w[(f * NP) / 32], (f * NP) % 32);
            const Real rho_lo = m[0] - var[0];
            Real mom2 = Real(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const Real mh = fabs(m[1 + a]) + var[1 + a];
                mom2 += mh * mh;
            }
            const Real e_lo = m[DIM + 1] - var[DIM + 1];
            // floors of Sec. 4.2 from the mean state (as below), and the margins
            const Real ke_bar = [&] {
                Real k = Real(0);
#pragma unroll
                for (int a = 0; a < DIM; ++a) k += m[1 + a] * m[1 + a];
                return k;
            }();
            const Real p_bar = (gam - Real(1)) * (m[DIM + 1] - Real(0.5) * ke_bar / m[0]);
            const Real tol = Real(1e-4);
            bool keep = m[0] > Real(0) && rho_lo - Real(1e-6) * m[0] > tol * (fabs(m[0]) + var[0]);
            if (keep) {
                const Real kin = Real(0.5) * mom2 / rho_lo;
                const Real p_lo = (gam - Real(1)) * (e_lo - kin);
                keep = p_lo - Real(1e-6) * p_bar > tol * (gam - Real(1)) * (fabs(m[DIM + 1]) + var[DIM + 1] + kin);
            }
            // the lanes' butterfly sums may differ in the last bit: lane 0 decides for the warp
            if (__shfl_sync(0xffffffffu, keep ? 1 : 0, 0)) continue;
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j)
            if (lane + 32 * j < NI) sM[lane + 32 * j] = w[j];
        __syncwarp();

        // widen axis 0, then 1 (then 2): Q -> E values per line
        {
            // pass x: sM [Q^d] -> sA [E * Q^(d-1)]
            constexpr int LX = NP / Q;
            for (int i = lane; i < NC * LX * E; i += 32) {
                const int r = i % E, fl = i / E;
                const Real *p = sM + fl * Q;
                Real acc = Real(0);
#pragma unroll
                for (int m = 0; m < Q; ++m) acc = fma(tE[r * Q + m], p[m], acc);
                sA[fl * E + r] = acc;
            }
            __syncwarp();
            // pass y: sA [E, Q, (Q)] -> sB [E, E, (Q)]
            constexpr int TZ = DIM == 3 ? Q : 1;
            for (int i = lane; i < NC * E * E * TZ; i += 32) {
                const int ix = i % E;
                const int ry = (i / E) % E;
                const int rest = i / (E * E);  // f * TZ + z
                const Real *p = sA + rest * (E * Q) + ix;
                Real acc = Real(0);
#pragma unroll
                for (int m = 0; m < Q; ++m) acc = fma(tE[ry * Q + m], p[m * E], acc);
                sB[rest * (E * E) + ry * E + ix] = acc;
            }
            __syncwarp();
            if (DIM == 3) {
                // pass z: sB [E, E, Q] -> sA [E, E, E]
                for (int i = lane; i < NC * NE; i += 32) {
                    const int ixy = i % (E * E);
                    const int rz = (i / (E * E)) % E;
                    const int f = i / NE;
                    const Real *p = sB + f * (E * E * Q) + ixy;
                    Real acc = Real(0);
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc = fma(tE[rz * Q + m], p[m * E * E], acc);
                    sA[f * NE + rz * E * E + ixy] = acc;
                }
                __syncwarp();
            }
        }
        const Real *pts = DIM == 3 ? sA : sB;  // [NC][NE] values on the widened grid

        const Real gamma = (Real)A.gamma;
        Real mean[NC];
#pragma unroll
        for (int f = 0; f < NC; ++f) mean[f] = sM[f * NP];
        Real rb, vb[3], pbar, cb;
        const bool ok_mean = primitives<DIM>(mean, gamma, rb, vb, pbar, cb);
        const Real rho_b = Real(1e-6) * mean[0], p_b = Real(1e-6) * pbar;

        // a point of the widened grid is used when at most one coordinate is at +-1
        auto used = [&](int i) {
            const int c0 = i % E, c1 = (i / E) % E, c2 = DIM == 3 ? i / (E * E) : 0;
            return (c0 >= Q) + (c1 >= Q) + (c2 >= Q) <= 1;
        };
        Real rmin = Real(1e30);
        for (int i = lane; i < NE; i += 32)
            if (used(i)) rmin = fmin(rmin, pts[i]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, off));
        const Real theta = rmin < rho_b ? (mean[0] - rho_b) / (mean[0] - rmin) : Real(1);

        int kmax = 0;
        bool fail = false;
        for (int i = lane; i < NE; i += 32) {
            if (!used(i)) continue;
            Real dv[NC];
#pragma unroll
            for (int f = 0; f < NC; ++f) dv[f] = pts[f * NE + i] - mean[f];
            int k = 0;
            for (; k <= 60; ++k) {
                const Real s = ldexp(theta, -k);
                Real u[NC];
#pragma unroll
                for (int f = 0; f < NC; ++f) u[f] = mean[f] + s * dv[f];
                Real ke = Real(0);
#pragma unroll
                for (int a = 0; a < DIM; ++a) ke += u[1 + a] * u[1 + a];
                const Real p = (gamma - Real(1)) * (u[DIM + 1] - Real(0.5) * ke / u[0]);
                if (p >= p_b) break;
            }
            if (k > 60) {
                fail = true;
                k = 60;
            }
            kmax = max(kmax, k);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, off));
        fail = __any_sync(0xffffffffu, fail);
        if (lane == 0 && (!ok_mean || fail)) atomicOr(A.status, DG_STATUS_NONPHYS);
        if (!ok_mean || (theta == Real(1) && kmax == 0)) continue;

        const Real sc = ldexp(theta, -kmax);
        for (int i = lane; i < NC * NP; i += 32) {
            const int f = i / NP, l = i % NP;
            const int sl = A.cmap ? A.cmap[l] : l;
            if (l == 0 || sl < 0) continue;
            const size_t gi = ((size_t)f * A.ncell + cell) * ms + sl;
            if (LAST) {
                const double u = A.ufull[gi] * (double)sc;
                A.ufull[gi] = u;
                if (A.uhi) A.uhi[gi] = (float)u;
            } else {
                // limited stage state sc * (u_base + delta), expressed as a new delta over u_base
                dl[gi] = sc * sM[i] - ub[gi];
            }
        }
    }
}

template <int DIM, int N, typename Real, bool TR>
cudaError_t run_limiter(const LimiterArgs &a, const Tables<Real> &t, cudaStream_t s)
{
    using PL = LimiterPlan<DIM, N, Real, TR>;
    auto k0 = limiter_kernel<DIM, N, Real, TR, false>;
    auto k1 = limiter_kernel<DIM, N, Real, TR, true>;
    // both variants are set up on every call (once per device), so the zero-cell launch that handles
    // make at creation prepares the one that the first step's limiter of u^{n+1} uses as well
    static KernelSetup ks[2];
    int sms = 0, bps[2] = {0, 0};
    cudaError_t e = kernel_setup(ks[0], k0, 32 * PL::CPB, PL::BYTES, &sms, &bps[0]);
    if (e != cudaSuccess) return e;
    e = kernel_setup(ks[1], k1, 32 * PL::CPB, PL::BYTES, &sms, &bps[1]);
    if (e != cudaSuccess) return e;
    auto k = a.last ? k1 : k0;
    const int bpsm = bps[a.last ? 1 : 0];
    if (a.ncell == 0) return cudaSuccess;
    // one wave of resident CTAs (persistent warps), fewer when the grid has fewer cells
    const long long need = (a.ncell + PL::CPB - 1) / PL::CPB;
    const long long blocks = need < (long long)sms * bpsm ? need : (long long)sms * bpsm;
    k<<<(unsigned)blocks, 32 * PL::CPB, PL::BYTES, s>>>(a, t);
    return cudaGetLastError();
}

template <int DIM, int N, typename Real>
cudaError_t run_limiter_any(const LimiterArgs &a, const Tables<Real> &t, cudaStream_t s)
{
    return a.tracer_on ? run_limiter<DIM, N, Real, true>(a, t, s) : run_limiter<DIM, N, Real, false>(a, t, s);
}

}  // namespace dgx
