// Persistent, line-oriented fused right-hand-side / Runge-Kutta stage kernel.
//
// The arithmetic is the collocated rewriting of the modal sums of Eq. time_stepping_final
// described in dgx_kernels.cuh; its organisation for sm_103a:
//  * one CTA loops over tiles. Plans with prefetch buffers stream the state of tile k+1 (u^n and
//    delta, tile + halo) into shared memory with cp.async while the CTA works on tile k; plans
//    without them (2-D FP32, two resident CTAs per SM) load a tile synchronously, straight into
//    registers, with the first modal->nodal pass applied before the only shared-memory store,
//    and rely on the other resident CTA to cover the load latency;
//  * the field count and the Navier-Stokes / artificial-viscosity switches are template
//    parameters, so every field loop unrolls;
//  * the modal<->nodal transforms work on whole lines of n+1 values: a thread reads its line
//    once into registers and writes the transformed line back in place (no second buffer, no
//    (n+1)-fold re-reads of shared memory);
//  * the last transposed pass (along x, where modes are contiguous) is fused with the
//    Runge-Kutta epilogue and writes each line of modes with one vector store.
#pragma once

#include <type_traits>

#include "dgx_kernels.cuh"

namespace dgx {

__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int DIM, int N, typename Real, bool AV, int NSM, int TX, int TY, int TZ, bool PF>
struct Stage2Plan {
    using S = Shape<DIM, N, TX, TY, TZ>;
    // NSM: physical diffusive fluxes -- 0 none, 1 Navier-Stokes (Sec. 3.3), 2 Navier-Stokes with a
    // passive tracer (Sec. 3.4, conserved field after the energy, whose diffusion needs the gradients)
    static constexpr bool NS = NSM >= 1;
    static constexpr bool TR = NSM == 2;
    // threads per CTA and the resident CTAs per SM the registers are bounded for (measured at
    // every degree): 2-D FP32 tiles balance their phases better over 10 warps (the 304 face
    // points of an 8x4 or 4x8 tile fit one round), 2 CTAs per SM; a 3-D FP32 tile fills most of
    // the shared memory, so one CTA per SM runs 16 warps to hide latency; FP64 uses 8 warps
    static constexpr int NTH = sizeof(Real) == 4 ? (DIM == 2 ? 320 : 512) : 256;
    static constexpr int MINB = (DIM == 2 && sizeof(Real) == 4) ? 2 : 1;
    static constexpr int Q = S::Q, NP = S::NP, NPF = S::NPF, NC = S::NC + (TR ? 1 : 0);
    static constexpr int NF = NC + (AV ? 1 : 0);
    static constexpr int TC = S::TC, NSLOT = S::NSLOT, NFACE = S::NFACE;
    static constexpr int TAB = (3 * Q * Q + 7 * Q + 1 + 3) / 4 * 4;
    // per-cell stride of the cell arrays in shared memory: one 16-byte unit more than a cell's
    // values when those fill whole units, so that the strided (y, z) line accesses of the cells
    // a warp touches spread over the banks; vector line accesses stay aligned
    static constexpr int NPS = NP + ((NP * (int)sizeof(Real)) % 16 == 0 ? 16 / (int)sizeof(Real) : 0);
    static constexpr int U16 = 16 / (int)sizeof(Real);  // values per 16 bytes; arrays are whole units
    static constexpr int SZ_IN = PF ? (NF * NSLOT * NPS + U16 - 1) / U16 * U16 : 0;  // u^n or delta, tile + halo
    static constexpr int SZ_U = (NF * NSLOT * NPS + U16 - 1) / U16 * U16;
    static constexpr int SZ_F = (DIM * NC * TC * NPS + U16 - 1) / U16 * U16;
    static constexpr int SZ_R = (NF * TC * NPS + U16 - 1) / U16 * U16;
    static constexpr int SZ_UT = NS ? NC * NFACE * NPF : 0;
    static constexpr int SZ_FH = NC * NFACE * NPF;
    static constexpr int OFF_IN0 = TAB;
    static constexpr int OFF_IN1 = OFF_IN0 + SZ_IN;
    static constexpr int OFF_U = OFF_IN1 + SZ_IN;
    static constexpr int OFF_F = OFF_U + SZ_U;
    static constexpr int OFF_R = OFF_F + SZ_F;
    static constexpr int OFF_UT = OFF_R + SZ_R;
    static constexpr int OFF_FH = OFF_UT + SZ_UT;
    static constexpr int OFF_WIG = OFF_FH + SZ_FH;
    static constexpr int NREAL = (OFF_WIG + TC + 3) / 4 * 4;
    static constexpr size_t BYTES = sizeof(Real) * (size_t)NREAL + sizeof(int) * 2 * (size_t)NSLOT;
    // bytes of one cell's modes of one field; async copies use the widest legal chunk
    static constexpr int CELL_BYTES = NP * (int)sizeof(Real);
    static constexpr int CHUNK = CELL_BYTES % 16 == 0 ? 16 : (CELL_BYTES % 8 == 0 ? 8 : 4);
    // widest access to one x-line of Q contiguous values (line starts are multiples of Q values
    // from a cell start, cell starts multiples of NPS values from an array start)
    static constexpr int LINE_BYTES = Q * (int)sizeof(Real);
    static constexpr int VEC = LINE_BYTES % 16 == 0 ? 16 : (LINE_BYTES % 8 == 0 ? 8 : (int)sizeof(Real));
    static_assert((NPS * (int)sizeof(Real)) % VEC == 0, "cell stride breaks line alignment");
    static_assert((OFF_IN0 * (int)sizeof(Real)) % 16 == 0 && (OFF_IN1 * (int)sizeof(Real)) % 16 == 0 &&
                      (OFF_U * (int)sizeof(Real)) % 16 == 0 && (OFF_R * (int)sizeof(Real)) % 16 == 0,
                  "cell arrays must start on 16-byte boundaries");
};

// the Q values of a cell along axis A starting at p (stride S): one vector access along x
template <int A, int Q, int VEC, int S, typename T>
__device__ __forceinline__ void ld_axis_line(const T *p, T (&w)[Q]);

// one x-line of Q contiguous values from / to shared or global memory with the widest aligned
// accesses (VEC bytes; the caller guarantees VEC alignment of p)
template <int Q, int VEC, typename T>
__device__ __forceinline__ void ld_line(const T *p, T (&w)[Q])
{
    if constexpr (VEC == 16 && sizeof(T) == 4) {
#pragma unroll
        for (int m = 0; m < Q; m += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p + m);
            w[m] = v.x;
            w[m + 1] = v.y;
            w[m + 2] = v.z;
            w[m + 3] = v.w;
        }
    } else if constexpr (VEC >= 8 && sizeof(T) == 4) {
#pragma unroll
        for (int m = 0; m < Q; m += 2) {
            const float2 v = *reinterpret_cast<const float2 *>(p + m);
            w[m] = v.x;
            w[m + 1] = v.y;
        }
    } else if constexpr (VEC == 16 && sizeof(T) == 8) {
#pragma unroll
        for (int m = 0; m < Q; m += 2) {
            const double2 v = *reinterpret_cast<const double2 *>(p + m);
            w[m] = v.x;
            w[m + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int m = 0; m < Q; ++m) w[m] = p[m];
    }
}

template <int A, int Q, int VEC, int S, typename T>
__device__ __forceinline__ void ld_axis_line(const T *p, T (&w)[Q])
{
    if constexpr (A == 0) {
        ld_line<Q, VEC>(p, w);
    } else {
#pragma unroll
        for (int m = 0; m < Q; ++m) w[m] = p[m * S];
    }
}

template <int Q, int VEC, typename T>
__device__ __forceinline__ void st_line(T *p, const T (&w)[Q])
{
    if constexpr (VEC == 16 && sizeof(T) == 4) {
#pragma unroll
        for (int m = 0; m < Q; m += 4) *reinterpret_cast<float4 *>(p + m) = make_float4(w[m], w[m + 1], w[m + 2], w[m + 3]);
    } else if constexpr (VEC >= 8 && sizeof(T) == 4) {
#pragma unroll
        for (int m = 0; m < Q; m += 2) *reinterpret_cast<float2 *>(p + m) = make_float2(w[m], w[m + 1]);
    } else if constexpr (VEC == 16 && sizeof(T) == 8) {
#pragma unroll
        for (int m = 0; m < Q; m += 2) *reinterpret_cast<double2 *>(p + m) = make_double2(w[m], w[m + 1]);
    } else {
#pragma unroll
        for (int m = 0; m < Q; ++m) p[m] = w[m];
    }
}

// Body shared by the single-simulation kernel (A0: its arguments) and the batched kernel (descs:
// one argument set per simulation; tile_off: prefix sums of the simulations' tile counts, so the
// work list is every (simulation, tile) pair in order).
template <int DIM, int N, typename Real, bool AV, int NSM, int TX, int TY, int TZ, bool PF, bool BATCH>
__device__ __forceinline__ void stage2_body(const StageArgs *A0, const StageArgs *descs, const int *tile_off,
                                            int nsims, const Tables<Real> &Tg)
{
    using S = Shape<DIM, N, TX, TY, TZ>;
    using PL = Stage2Plan<DIM, N, Real, AV, NSM, TX, TY, TZ, PF>;
    constexpr int Q = S::Q, NP = S::NP, NPF = S::NPF, NC = PL::NC, TC = S::TC, NSLOT = S::NSLOT;
    constexpr bool NS = PL::NS, TR = PL::TR;
    constexpr int NF = PL::NF, NFACE = S::NFACE, NPS = PL::NPS, VEC = PL::VEC;
    constexpr bool GRAD = AV || NS;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *sm = reinterpret_cast<Real *>(smem_raw);
    Real *tB = sm, *tDn = tB + Q * Q, *tWd = tDn + Q * Q, *tG = tWd + Q * Q;
    Real *tLp = tG + Q, *tLm = tLp + Q, *tCm = tLm + Q, *tCp = tCm + Q, *tDm = tCp + Q, *tDp = tDm + Q;
    Real *sIn0 = sm + PL::OFF_IN0, *sIn1 = sm + PL::OFF_IN1, *sU = sm + PL::OFF_U, *sF = sm + PL::OFF_F;
    Real *sR = sm + PL::OFF_R, *sUt = sm + PL::OFF_UT, *sFh = sm + PL::OFF_FH, *sWig = sm + PL::OFF_WIG;
    __shared__ double s_red[2][PL::NTH / 32];
    int *sGa = reinterpret_cast<int *>(sm + PL::NREAL);
    int *sGb = sGa + NSLOT;
    __shared__ int s_status;

    // every launch uses PL::NTH threads: loop strides are compile-time constants, so the
    // per-thread loops unroll and their index arithmetic folds
    const int tid = threadIdx.x;
    constexpr int nth = PL::NTH;
    const int ntiles = BATCH ? tile_off[nsims] : A0->ntile[0] * A0->ntile[1] * A0->ntile[2];
    // simulation of a work-list tile (binary search in the prefix sums)
    auto sim_of = [&](int tile) -> int {
        if (!BATCH) return 0;
        int lo = 0, hi = nsims - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_off[mid] <= tile) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    auto args_of = [&](int sim) -> const StageArgs & { return BATCH ? descs[sim] : *A0; };
    auto local_tile = [&](int tile, int sim) { return BATCH ? tile - tile_off[sim] : tile; };

    for (int i = tid; i < Q * Q; i += nth) {
        tB[i] = Tg.B[i / Q][i % Q];
        tDn[i] = Tg.Dn[i / Q][i % Q];
        tWd[i] = Tg.Wd[i / Q][i % Q];
    }
    for (int i = tid; i < Q; i += nth) {
        tG[i] = Tg.G[i];
        tLp[i] = Tg.Lp[i];
        tLm[i] = Tg.Lm[i];
        tCm[i] = Tg.Cm[i];
        tCp[i] = Tg.Cp[i];
        tDm[i] = Tg.Dm[i];
        tDp[i] = Tg.Dp[i];
    }
    if (tid == 0) s_status = 0;

    // time step of the step from the first stage's per-CTA maxima (Eq. timestep), identical in
    // every CTA (maxima are exact in any order)
    __shared__ double s_dt;
    if (!BATCH && A0->dt_partial) {
        double c = 0.0, v = 0.0;
        for (int i = tid; i < A0->dt_nblk; i += nth) {
            c = fmax(c, A0->dt_partial[2 * i]);
            v = fmax(v, A0->dt_partial[2 * i + 1]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            c = fmax(c, __shfl_xor_sync(0xffffffffu, c, off));
            v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
        }
        if ((tid & 31) == 0) {
            s_red[0][tid >> 5] = c;
            s_red[1][tid >> 5] = v;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nth / 32; ++w) {
                c = fmax(c, s_red[0][w]);
                v = fmax(v, s_red[1][w]);
            }
            const double dt = A0->dt_fixed > 0.0 ? A0->dt_fixed : A0->cfl * A0->hmin / (2.0 * (N + 1) * (c + v));
            s_dt = dt;
            if (blockIdx.x == 0) {
                if (!(dt > 0.0) || !isfinite(dt)) atomicOr(A0->status, DG_STATUS_BADDT);
                double *dtp = const_cast<double *>(A0->dtp);
                dtp[0] = dt;
                dtp[1] += 1.0;
                dtp[2] += dt;
            }
        }
        __syncthreads();
    }

    auto tile_origin = [&](const StageArgs &T, int tile, int *o, int *V) {
        int b = tile;
        const int tx = b % T.ntile[0];
        b /= T.ntile[0];
        const int ty = b % T.ntile[1];
        const int tz = b / T.ntile[1];
        o[0] = tx * TX;
        o[1] = ty * TY;
        o[2] = tz * TZ;
        V[0] = min(TX, T.N[0] - o[0]);
        V[1] = min(TY, T.N[1] - o[1]);
        V[2] = DIM == 3 ? min(TZ, T.N[2] - o[2]) : 1;
    };

    // slot indices of a tile, then asynchronous copies of its stage state into sIn0 / sIn1
    // (called by all threads of the CTA)
    auto issue_tile = [&](const StageArgs &T, int tile, int *sG) {
        int o[3], V[3];
        tile_origin(T, tile, o, V);
        const Real *ub = static_cast<const Real *>(T.ubase);
        const Real *di = static_cast<const Real *>(T.din);
        for (int s = tid; s < NSLOT; s += nth) sG[s] = slot_global<S>(s, o, V, T.N, T.bc);
        __syncthreads();
        if constexpr (!PF) return;  // without prefetch buffers the tile is loaded (fused with pass A) at the top of its iteration
        constexpr int PER = PL::CELL_BYTES / PL::CHUNK;  // chunks per (field, cell)
        // one (slot, chunk) pair per thread and pass, all fields by a constant stride
        const size_t gfield = (size_t)T.ncell * NP * sizeof(Real);          // bytes between fields
        constexpr size_t sfield = (size_t)NSLOT * NPS * sizeof(Real);
        for (int p = tid; p < NSLOT * PER; p += nth) {
            const int slot = p / PER, c = p % PER;
            const int g = sG[slot];
            if (g < 0) continue;
            const char *gu = reinterpret_cast<const char *>(ub) + (size_t)g * NP * sizeof(Real) + (size_t)c * PL::CHUNK;
            char *su = reinterpret_cast<char *>(sIn0) + (size_t)slot * NPS * sizeof(Real) + (size_t)c * PL::CHUNK;
            const char *gd = di ? reinterpret_cast<const char *>(di) + (gu - reinterpret_cast<const char *>(ub)) : nullptr;
            char *sd = reinterpret_cast<char *>(sIn1) + (su - reinterpret_cast<char *>(sIn0));
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if (PL::CHUNK == 16) cp_async_16(su + f * sfield, gu + f * gfield);
                else if (PL::CHUNK == 8) cp_async_8(su + f * sfield, gu + f * gfield);
                else cp_async_4(su + f * sfield, gu + f * gfield);
                if (gd) {
                    if (PL::CHUNK == 16) cp_async_16(sd + f * sfield, gd + f * gfield);
                    else if (PL::CHUNK == 8) cp_async_8(sd + f * sfield, gd + f * gfield);
                    else cp_async_4(sd + f * sfield, gd + f * gfield);
                }
            }
        }
        cp_async_commit();
    };

    Real cmax = Real(0), vmax = Real(0);  // CFL speeds (fused first stage)
    int bad = 0;

    int tile = blockIdx.x;
    int *sG = sGa, *sGn = sGb;
    __syncthreads();
    if (tile < ntiles) {
        const int sim = sim_of(tile);
        issue_tile(args_of(sim), local_tile(tile, sim), sG);
    }

    // batched: the current simulation's arguments live in shared memory, so that the compiler need
    // not reload them from global memory after every global store of the tile
    __shared__ __align__(16) StageArgs s_desc;
    int s_sim = -1;
    while (tile < ntiles) {
        const int sim = sim_of(tile);
        if constexpr (BATCH) {
            if (sim != s_sim) {  // uniform over the CTA
                __syncthreads();  // the previous tile's last reads of s_desc are done
                const unsigned long long *src = reinterpret_cast<const unsigned long long *>(descs + sim);
                unsigned long long *dst = reinterpret_cast<unsigned long long *>(&s_desc);
                for (int i = tid; i < (int)(sizeof(StageArgs) / 8); i += nth) dst[i] = src[i];
                __syncthreads();
                s_sim = sim;
            }
        }
        const StageArgs &A = BATCH ? s_desc : *A0;
        int o[3], V[3];
        tile_origin(A, local_tile(tile, sim), o, V);
        const Real *ub = static_cast<const Real *>(A.ubase);
        const Real *di = static_cast<const Real *>(A.din);
        const Real *K;
        if constexpr (sizeof(Real) == 4) K = A.kf;
        else K = A.kd;
        const Real gamma = K[SK_GAMMA], nu = K[SK_NU], kappa = K[SK_KAPPA], eta = K[SK_ETA];
        const Real epsfac = K[SK_EPS], inv_tau = K[SK_INV_TAU], f_v = K[SK_FV];
        const Real inv_f = Tg.inv_f;
        Real two_h[3], cax[3], inv_h[3];
    #pragma unroll
        for (int a = 0; a < 3; ++a) {
            two_h[a] = K[SK_TWO_H + a];
            inv_h[a] = K[SK_INV_H + a];
            cax[a] = K[SK_CAX + a];
        }
        const Real src_w = (Real)(DIM == 2 ? 0.25 : 0.125);
        const double dstep = (!BATCH && A.dt_partial) ? s_dt : (A.dtp ? A.dtp[0] : 0.0);
        const Real dt = A.epi_unit_dt ? Real(1) : (A.mode != 0 ? (Real)dstep : Real(0));
        const Real dsc = A.din_dt ? (Real)(A.din_coef * dstep) : Real(1);  // stored delta -> true delta
        const Real ca = K[SK_CA], cx = K[SK_CX], cb = K[SK_CB];
        const Real za = K[SK_ZA], zx = K[SK_ZX], zb = K[SK_ZB];
        Real *xb = static_cast<Real *>(A.xbuf);
        Real *dout = static_cast<Real *>(A.dout);
        const bool readx = xb && (A.cx != 0.0 || A.zx != 0.0);

        if constexpr (PF) {
            cp_async_wait_all();
            __syncthreads();
        } else {
            // synchronous load of u^n (+ delta) of tile and halo fused with pass A (x-lines, modal ->
            // nodal): one (slot, x-line) per thread and pass, all fields by a constant stride so that
            // their loads are in flight together, transformed in registers and stored as nodal values;
            // the modal density of the tile's own cells is kept in sR (free until the volume phase) for
            // the sensor of the fused first stage
            constexpr int LPC = NP / Q;  // x-lines per cell
            const bool keep = AV && A.fused;
            for (int p = tid; p < NSLOT * LPC; p += nth) {
                const int slot = p / LPC, r = p % LPC;
                const int g = sG[slot];
                if (g < 0) continue;
                // library-owned arrays: a line starts at a multiple of Q values, so VEC accesses are legal
                const size_t g0 = (size_t)g * NP + (size_t)r * Q;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const size_t gi = g0 + (size_t)f * A.ncell * NP;
                    Real w[Q];
                    ld_line<Q, VEC>(ub + gi, w);
                    if (di) {
                        Real dd[Q];
                        ld_line<Q, VEC>(di + gi, dd);
#pragma unroll
                        for (int m = 0; m < Q; ++m) w[m] = w[m] + dsc * dd[m];
                    }
                    if (f == 0 && keep && slot < TC) st_line<Q, VEC>(sR + slot * NPS + r * Q, w);
                    Real o[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        Real acc = Real(0);
#pragma unroll
                        for (int m = 0; m < Q; ++m) acc = fma(Tg.B[i][m], w[m], acc);
                        o[i] = acc;
                    }
                    st_line<Q, VEC>(sU + (f * NSLOT + slot) * NPS + r * Q, o);
                }
            }
            __syncthreads();
        }
        // wiggle source per tile cell: from the sensor of u^n (fused first stage) or as stored
        auto cell_wiggle = [&](const Real *modal) {
            for (int c = tid; c < TC; c += nth) {
                const int g = sG[c];
                if (g < 0) continue;
                if (!A.fused) {
                    sWig[c] = (Real)A.wig[g];
                    continue;
                }
                Real hi = Real(0), all = Real(0);
                const Real *w0 = modal + c * NPS;  // density field, slot c
#pragma unroll
                for (int l = 0; l < NP; ++l) {
                    const int l0 = l % Q, l1 = (l / Q) % Q, l2 = DIM == 3 ? l / (Q * Q) : 0;
                    // the modes the degree-(n-1) basis lacks (Sec. 4.1)
                    const bool top = N > 0 && (A.total_degree ? (l0 + l1 + l2 == N)
                                                              : (l0 == N || l1 == N || (DIM == 3 && l2 == N)));
                    all += w0[l] * w0[l];
                    if (top) hi += w0[l] * w0[l];
                }
                const double Sk = all > Real(0) ? (double)(hi / all) : 0.0;
                const double dt_prev = A.dtp[0], step = A.dtp[1];
                const double s_floor = 1e-4 * A.s_on;
                double dlog = 0.0;
                if (step > 0.0 && dt_prev > 0.0) {
                    if constexpr (sizeof(Real) == 4) {
                        // the sensor of the FP32 modes carries FP32 precision: take its logarithm in FP32
                        // (FP64 arithmetic is a small fraction of the FP32 rate on this part)
                        const float sf = (float)s_floor;
                        dlog = (double)((logf(fmaxf((float)Sk, sf)) - logf(fmaxf((float)A.S_prev[g], sf))) /
                                        (float)dt_prev);
                    } else {
                        dlog = (log(fmax(Sk, s_floor)) - log(fmax(A.S_prev[g], s_floor))) / dt_prev;
                    }
                }
                const double wg = (Sk > A.s_on) ? A.f_w * fmax(0.0, dlog) : 0.0;
                A.wig_w[g] = wg;
                A.S_prev[g] = Sk;
                sWig[c] = (Real)wg;
            }
        };
        // (the barrier after pass B orders these reads and the sWig writes before the volume phase)
        if (AV) {
            if constexpr (PF) cell_wiggle(sIn0);  // the modal u^n stays in sIn0 during pass A (first stage: no delta)
            else cell_wiggle(sR);
        }

        // ---- pass A: x-lines, modal -> nodal, from the loaded input (u^n + delta); without prefetch
        // buffers it is part of the load above
        if constexpr (PF) {
            constexpr int LINES = NF * NSLOT * (NP / Q);
            for (int idx = tid; idx < LINES; idx += nth) {
                const int fs = idx / (NP / Q);
                const int r = idx % (NP / Q);
                if (sG[fs % NSLOT] < 0) continue;
                const int base = fs * NPS + r * Q;
                Real w[Q];
                ld_line<Q, VEC>(sIn0 + base, w);
                if (di) {
                    Real dd[Q];
                    ld_line<Q, VEC>(sIn1 + base, dd);
#pragma unroll
                    for (int m = 0; m < Q; ++m) w[m] = fma(dsc, dd[m], w[m]);
                }
                Real o[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    Real acc = Real(0);
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc = fma(Tg.B[i][m], w[m], acc);
                    o[i] = acc;
                }
                st_line<Q, VEC>(sU + base, o);
            }
            __syncthreads();
        }
        // the input buffers are free: start streaming the next tile
        const int next = tile + gridDim.x;
        if (PF && next < ntiles) {
            const int nsim = sim_of(next);
            issue_tile(args_of(nsim), local_tile(next, nsim), sGn);
        }

        // ---- passes B (y) and C (z) in place
#pragma unroll
        for (int a = 1; a < DIM; ++a) {
            const int Sa = S::S(a);
            constexpr int LINES = NF * NSLOT * (NP / Q);
            for (int idx = tid; idx < LINES; idx += nth) {
                const int fs = idx / (NP / Q);
                const int r = idx % (NP / Q);
                if (sG[fs % NSLOT] < 0) continue;
                // r enumerates the (Q^(d-1)) positions transverse to axis a
                const int lo = r % Sa, hi = r / Sa;
                const int base = fs * NPS + lo + hi * Sa * Q;
                Real w[Q];
#pragma unroll
                for (int m = 0; m < Q; ++m) w[m] = sU[base + m * Sa];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    Real acc = Real(0);
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc = fma(Tg.B[i][m], w[m], acc);
                    sU[base + i * Sa] = acc;
                }
            }
            __syncthreads();
        }

        // ---- pointwise volume fluxes and alpha source; recovered interface state (NS)
        {
            constexpr int NODES = TC * NP;
            for (int idx = tid; idx < NODES; idx += nth) {
                const int c = idx / NP, j = idx % NP;
                const int g = sG[c];
                if (g < 0) continue;
                Real u[NC + 1];
#pragma unroll
                for (int f = 0; f < NF; ++f) u[f] = sU[(f * NSLOT + c) * NPS + j];
                Real gr[DIM][NC];
                if (GRAD) {
#pragma unroll
                    for (int a = 0; a < DIM; ++a) {
                        const int Sa = S::S(a);
                        const int i = (j / Sa) % Q;
                        const int base = j - i * Sa;
#pragma unroll
                        for (int f = 0; f < NC; ++f) {
                            const Real *p = sU + (f * NSLOT + c) * NPS + base;
                            Real acc = Real(0);
#pragma unroll
                            for (int m = 0; m < Q; ++m) acc = fma(tDn[i * Q + m], p[m * Sa], acc);
                            gr[a][f] = acc * two_h[a];
                        }
                    }
                }
                Real rho, v[3], p, cs;
                if (!primitives<DIM>(u, gamma, rho, v, p, cs)) bad = 1;
                if (A.fused) {
                    Real v2 = Real(0);
#pragma unroll
                    for (int a = 0; a < DIM; ++a) v2 += v[a] * v[a];
                    cmax = fmax(cmax, cs);
                    vmax = fmax(vmax, sqrt(v2));
                }
                const Real eps = AV ? epsfac * clamp01(u[NC]) * cs : Real(0);
                const int jj[3] = {j % Q, (j / Q) % Q, j / (Q * Q)};
                Real Gv = Real(1);
#pragma unroll
                for (int a = 0; a < DIM; ++a) Gv *= tG[jj[a]];
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    Real F[NC];
                    euler_flux<DIM, TR>(u, v, p, a, F);
                    if (NS) {
                        Real Fn[NC];
                        ns_flux<DIM, TR>(u, gr, gamma, nu, kappa, eta, a, Fn);
#pragma unroll
                        for (int f = 0; f < NC; ++f) F[f] -= Fn[f];
                    }
                    if (AV) {
#pragma unroll
                        for (int f = 0; f < NC; ++f) F[f] -= eps * gr[a][f];
                    }
                    Real Gp = Real(1);
#pragma unroll
                    for (int q = 0; q < DIM; ++q)
                        if (q != a) Gp *= tG[jj[q]];
                    const Real w = cax[a] * Gp;
#pragma unroll
                    for (int f = 0; f < NC; ++f) sF[((a * NC + f) * TC + c) * NPS + j] = w * F[f];
                }
                if (A.force) {
                    // driving source of Sec. 7.1 at this node, Gauss-weighted like the alpha source:
                    // rho s into the momentum, s.(rho v) into the energy; the conserved part of sR
                    // is free until the residual phase, which adds it
                    const Real *fs = static_cast<const Real *>(A.force);
                    const Real wgt = src_w * Gv;
                    Real se = Real(0);
#pragma unroll
                    for (int a = 0; a < DIM; ++a) {
                        const Real sa = fs[((size_t)a * A.ncell + g) * NP + j];
                        sR[((1 + a) * TC + c) * NPS + j] = wgt * u[0] * sa;
                        se = fma(sa, u[1 + a], se);
                    }
                    sR[((DIM + 1) * TC + c) * NPS + j] = wgt * se;
                }
                if (AV) {
                    Real div = Real(0);
#pragma unroll
                    for (int a = 0; a < DIM; ++a) div += (gr[a][1 + a] - v[a] * gr[a][0]) / rho;
                    const Real adot = f_v * fmax(Real(0), -div) + sWig[c] - u[NC] * cs * inv_tau;
                    sR[(NC * TC + c) * NPS + j] = src_w * Gv * adot;
                }
            }
            if (NS) {
                // recovered state at every face point, one loop per axis with the axis known at compile time
                auto recover_axis = [&](auto axc) {
                    constexpr int a = decltype(axc)::value;
                    constexpr int Sa = S::S(a);
                    constexpr int FA = S::NFA(a);
                    for (int q = tid; q < NC * FA * NPF; q += nth) {
                        const int k = q % NPF;
                        const int fc = q / NPF;
                        const int fl = fc % FA, f = fc / FA;
                        const int pp = fl % (S::T(a) + 1);
                        const int t = fl / (S::T(a) + 1);
                        int cc[3] = {0, 0, 0};
                        S::untrans(a, t, cc);
                        bool ok = pp <= V[a];
#pragma unroll
                        for (int b2 = 0; b2 < 3; ++b2)
                            if (b2 != a && cc[b2] >= V[b2]) ok = false;
                        if (!ok) continue;
                        int cl[3] = {cc[0], cc[1], cc[2]}, cr[3] = {cc[0], cc[1], cc[2]};
                        cl[a] = pp - 1;
                        cr[a] = pp;
                        const int sl = pp > 0 ? cl[0] + TX * (cl[1] + TY * cl[2]) : S::HOFF(a, 0) + t;
                        const int sr = pp < V[a] ? cr[0] + TX * (cr[1] + TY * cr[2]) : S::HOFF(a, 1) + t;
                        if (sG[sl] < 0 || sG[sr] < 0) continue;
                        const int base = S::knode(a, 0, k);
                        Real lv[Q], rv[Q];
                        ld_axis_line<a, Q, VEC, Sa>(sU + (f * NSLOT + sl) * NPS + base, lv);
                        ld_axis_line<a, Q, VEC, Sa>(sU + (f * NSLOT + sr) * NPS + base, rv);
                        Real acc = Real(0);
#pragma unroll
                        for (int m = 0; m < Q; ++m) acc = fma(Tg.Cm[m], lv[m], fma(Tg.Cp[m], rv[m], acc));
                        sUt[(f * NFACE + S::FOFF(a) + fl) * NPF + k] = acc;
                    }
                };
                recover_axis(std::integral_constant<int, 0>{});
                recover_axis(std::integral_constant<int, 1>{});
                if constexpr (DIM == 3) recover_axis(std::integral_constant<int, 2>{});
            }
        }
        __syncthreads();

        // ---- face fluxes (HLLC - recovered dissipative flux), pre-weighted for the lift
        auto flux_axis = [&](auto axc) {
          constexpr int a = decltype(axc)::value;
          constexpr int FA = S::NFA(a);
          for (int idx = tid; idx < FA * NPF; idx += nth) {
            const int k = idx % NPF, fl = idx / NPF;
            const int face = S::FOFF(a) + fl;
            const int pp = fl % (S::T(a) + 1);
            const int t = fl / (S::T(a) + 1);
            int cc[3] = {0, 0, 0};
            S::untrans(a, t, cc);
            bool ok = pp <= V[a];
#pragma unroll
            for (int b2 = 0; b2 < 3; ++b2)
                if (b2 != a && cc[b2] >= V[b2]) ok = false;
            if (!ok) continue;
            int cl[3] = {cc[0], cc[1], cc[2]}, cr[3] = {cc[0], cc[1], cc[2]};
            cl[a] = pp - 1;
            cr[a] = pp;
            const int sl = pp > 0 ? cl[0] + TX * (cl[1] + TY * cl[2]) : S::HOFF(a, 0) + t;
            const int sr = pp < V[a] ? cr[0] + TX * (cr[1] + TY * cr[2]) : S::HOFF(a, 1) + t;
            constexpr int Sa = S::S(a);
            const int base = S::knode(a, 0, k);
            Real Fh[NC];
            if (sG[sl] < 0 || sG[sr] < 0) {
                const bool right_in = sG[sl] < 0;
                const int si = right_in ? sr : sl;

                Real u[NC], v[3], rho, pr_, cs;
#pragma unroll
                for (int f = 0; f < NC; ++f) {
                    Real qv[Q];
                    ld_axis_line<a, Q, VEC, Sa>(sU + (f * NSLOT + si) * NPS + base, qv);
                    Real acc = Real(0);
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc = fma(right_in ? Tg.Lm[m] : Tg.Lp[m], qv[m], acc);
                    u[f] = acc;
                }
                if (!primitives<DIM>(u, gamma, rho, v, pr_, cs)) bad = 1;
                euler_flux<DIM, TR>(u, v, pr_, a, Fh);
            } else {
                // traces of both sides and, for the dissipative flux, the recovered normal derivative,
                // from one load of each side's line normal to the face
                Real uL[NC + 1], uR[NC + 1], dn[NC];
                const Real sc = inv_f * inv_h[a];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    Real lv[Q], rv[Q];
                    ld_axis_line<a, Q, VEC, Sa>(sU + (f * NSLOT + sl) * NPS + base, lv);
                    ld_axis_line<a, Q, VEC, Sa>(sU + (f * NSLOT + sr) * NPS + base, rv);
                    Real al = Real(0), ar = Real(0);
#pragma unroll
                    for (int m = 0; m < Q; ++m) {
                        al = fma(Tg.Lp[m], lv[m], al);
                        ar = fma(Tg.Lm[m], rv[m], ar);
                    }
                    uL[f] = al;
                    uR[f] = ar;
                    if (GRAD && f < NC) {
                        Real acc = Real(0);
#pragma unroll
                        for (int m = 0; m < Q; ++m) acc = fma(Tg.Dm[m], lv[m], fma(Tg.Dp[m], rv[m], acc));
                        dn[f] = acc * sc;
                    }
                }
                Real cL, cR;  // trace sound speeds, reused by the artificial viscosity below
                if (!hllc<DIM, TR>(uL, uR, gamma, a, Fh, cL, cR)) bad = 1;
                if (GRAD) {
                    if (NS) {
                        Real ut[NC], grd[DIM][NC];
                        const int k0 = k % Q, k1 = k / Q;
#pragma unroll
                        for (int f = 0; f < NC; ++f) {
                            const Real *pf = sUt + (f * NFACE + face) * NPF;
                            ut[f] = pf[k];
#pragma unroll
                            for (int bb = 0; bb < DIM; ++bb) grd[bb][f] = Real(0);
                            grd[a][f] = dn[f];
                            int tb = 0;
#pragma unroll
                            for (int bb = 0; bb < DIM; ++bb) {
                                if (bb == a) continue;
                                const int kb = tb == 0 ? k0 : k1;
                                const int sb = tb == 0 ? 1 : Q;
                                const Real *q = pf + (k - kb * sb);
                                Real acc = Real(0);
#pragma unroll
                                for (int m = 0; m < Q; ++m) acc = fma(tDn[kb * Q + m], q[m * sb], acc);
                                grd[bb][f] = acc * two_h[bb];
                                ++tb;
                            }
                        }
                        if (!(ut[0] > Real(0))) bad = 1;
                        Real Fn[NC];
                        ns_flux<DIM, TR>(ut, grd, gamma, nu, kappa, eta, a, Fn);
#pragma unroll
                        for (int f = 0; f < NC; ++f) Fh[f] -= Fn[f];
                    }
                    if (AV) {
                        const Real eps = Real(0.5) * epsfac * (clamp01(uL[NC]) * cL + clamp01(uR[NC]) * cR);
#pragma unroll
                        for (int f = 0; f < NC; ++f) Fh[f] -= eps * dn[f];
                    }
                }
            }
            Real Gp = tG[k % Q];
            if (DIM == 3) Gp *= tG[k / Q];
            const Real w = cax[a] * Gp;
#pragma unroll
            for (int f = 0; f < NC; ++f) sFh[(f * NFACE + face) * NPF + k] = w * Fh[f];
          }
        };
        flux_axis(std::integral_constant<int, 0>{});
        flux_axis(std::integral_constant<int, 1>{});
        if constexpr (DIM == 3) flux_axis(std::integral_constant<int, 2>{});
        __syncthreads();

        // ---- nodal residual of the conserved fields: weak divergence + lift, one pass per axis over
        // the lines of Q nodes along it, all Q outputs of a line at once (the operator tables are
        // kernel-parameter operands); the first pass starts from the driving source, if any, the
        // later ones add to the stored partial sums
        auto residual_axis = [&](auto axc) {
            constexpr int a = decltype(axc)::value;
            constexpr int Sa = S::S(a);
            constexpr int LPC = NP / Q;  // lines per cell along a = face points per face
            for (int idx = tid; idx < NC * TC * LPC; idx += nth) {
                const int k = idx % LPC;  // transverse node in the face numbering
                const int fc = idx / LPC;
                const int c = fc % TC, f = fc / TC;
                if (sG[c] < 0) continue;
                const int cx = c % TX, cy = (c / TX) % TY, cz = c / (TX * TY);
                const int ca = a == 0 ? cx : (a == 1 ? cy : cz);
                const int fl = S::FOFF(a) + ca + (S::T(a) + 1) * S::trans(a, cx, cy, cz);
                const Real fL = sFh[(f * NFACE + fl) * NPF + k];
                const Real fR = sFh[(f * NFACE + fl + 1) * NPF + k];
                const int n0 = S::knode(a, 0, k);
                const Real *Fp = sF + ((a * NC + f) * TC + c) * NPS + n0;
                Real *rp = sR + fc * NPS + n0;
                Real F[Q], r[Q];
                if constexpr (a == 0) {
                    ld_line<Q, VEC>(Fp, F);
                    if (A.force && f > 0 && f <= DIM + 1) {  // momentum and energy
                        ld_line<Q, VEC>(rp, r);
                    } else {
#pragma unroll
                        for (int i = 0; i < Q; ++i) r[i] = Real(0);
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < Q; ++m) {
                        F[m] = Fp[m * Sa];
                        r[m] = rp[m * Sa];
                    }
                }
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    Real acc = r[i];
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc = fma(Tg.Wd[i][m], F[m], acc);
                    acc = fma(Tg.Lm[i], fL, acc);
                    r[i] = fma(-Tg.Lp[i], fR, acc);
                }
                if constexpr (a == 0) {
                    st_line<Q, VEC>(rp, r);
                } else {
#pragma unroll
                    for (int i = 0; i < Q; ++i) rp[i * Sa] = r[i];
                }
            }
        };
        residual_axis(std::integral_constant<int, 0>{});
        __syncthreads();
        residual_axis(std::integral_constant<int, 1>{});
        if constexpr (DIM == 3) {
            __syncthreads();
            residual_axis(std::integral_constant<int, 2>{});
        }
        __syncthreads();

        // ---- nodal -> modal: transposed passes along z and y in place
#pragma unroll
        for (int a = DIM - 1; a >= 1; --a) {
            const int Sa = S::S(a);
            constexpr int LINES = NF * TC * (NP / Q);
            for (int idx = tid; idx < LINES; idx += nth) {
                const int fc = idx / (NP / Q);
                const int r = idx % (NP / Q);
                if (sG[fc % TC] < 0) continue;
                const int lo = r % Sa, hi = r / Sa;
                const int base = fc * NPS + lo + hi * Sa * Q;
                Real w[Q];
#pragma unroll
                for (int m = 0; m < Q; ++m) w[m] = sR[base + m * Sa];
#pragma unroll
                for (int l = 0; l < Q; ++l) {
                    Real acc = Real(0);
#pragma unroll
                    for (int i = 0; i < Q; ++i) acc = fma(Tg.B[i][l], w[i], acc);
                    sR[base + l * Sa] = acc;
                }
            }
            __syncthreads();
        }

        // ---- last transposed pass along x fused with the Runge-Kutta epilogue
        {
            constexpr int LINES = NF * TC * (NP / Q);
            for (int idx = tid; idx < LINES; idx += nth) {
                const int fc = idx / (NP / Q);
                const int r = idx % (NP / Q);
                const int c = fc % TC, f = fc / TC;
                const int g = sG[c];
                if (g < 0) continue;
                const int base = fc * NPS + r * Q;
                const size_t gi = ((size_t)f * A.ncell + g) * NP + (size_t)r * Q;
                // library-owned arrays: a line starts at a multiple of Q values, so the widest
                // aligned access of the line's bytes is legal
                constexpr int VD = (Q * 8) % 16 == 0 ? 16 : 8;
                constexpr int VF = (Q * 4) % 16 == 0 ? 16 : ((Q * 4) % 8 == 0 ? 8 : 4);
                // u^n of the line is loaded before the transposed pass: the compiler may not move
                // the load past the earlier stores it cannot prove disjoint, and this way its latency
                // overlaps the arithmetic
                double uo[Q];
                if (A.mode == 2) ld_line<Q, VD>(A.uold + gi, uo);
                Real w[Q], L[Q];
                ld_line<Q, VEC>(sR + base, w);
#pragma unroll
                for (int l = 0; l < Q; ++l) {
                    Real acc = Real(0);
#pragma unroll
                    for (int i = 0; i < Q; ++i) acc = fma(Tg.B[i][l], w[i], acc);
                    L[l] = acc;
                }
                if (A.total_degree) {
                    // total-degree basis: modes with l_x + l_y + l_z > n are not in the space and stay 0
                    const int lyz = r % Q + (DIM == 3 ? r / Q : 0);
#pragma unroll
                    for (int l = 0; l < Q; ++l)
                        if (l + lyz > N) L[l] = Real(0);
                }
                if (A.mode == 0) {
#pragma unroll
                    for (int l = 0; l < Q; ++l) A.rhs_out[gi + l] = (double)L[l];
                    continue;
                }
                Real din[Q], xv[Q], dnew[Q], zn[Q];
                if (di) {
                    ld_line<Q, VEC>(di + gi, din);
#pragma unroll
                    for (int l = 0; l < Q; ++l) din[l] = dsc * din[l];
                } else {
#pragma unroll
                    for (int l = 0; l < Q; ++l) din[l] = Real(0);
                }
                if (readx) {
                    ld_line<Q, VEC>(xb + gi, xv);
                } else {
#pragma unroll
                    for (int l = 0; l < Q; ++l) xv[l] = Real(0);
                }
#pragma unroll
                for (int l = 0; l < Q; ++l) {
                    const Real dtL = dt * L[l];
                    dnew[l] = ca * din[l] + cx * xv[l] + cb * dtL;
                    zn[l] = za * din[l] + zx * xv[l] + zb * dtL;
                }
                if (A.write_z) st_line<Q, VEC>(xb + gi, zn);
                if (A.mode == 1) {
                    st_line<Q, VEC>(dout + gi, dnew);
                } else {
                    double un[Q];
#pragma unroll
                    for (int l = 0; l < Q; ++l) un[l] = uo[l] + (double)dnew[l];
                    st_line<Q, VD>(A.unew + gi, un);
                    if (A.uhi_new) {
                        float uf[Q];
#pragma unroll
                        for (int l = 0; l < Q; ++l) uf[l] = (float)un[l];
                        st_line<Q, VF>(A.uhi_new + gi, uf);
                    }
                }
            }
        }
        __syncthreads();
        if constexpr (PF) {
            int *t = sG;
            sG = sGn;
            sGn = t;
        } else if (next < ntiles) {
            const int nsim = sim_of(next);
            issue_tile(args_of(nsim), local_tile(next, nsim), sG);  // slot map of the next tile
        }
        if (BATCH) {
            // per-simulation results of this tile: CFL maxima (fused first stage) and status
            if (A.fused) {
                double c = (double)cmax, v = (double)vmax;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    c = fmax(c, __shfl_xor_sync(0xffffffffu, c, off));
                    v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
                }
                if ((tid & 31) == 0) {
                    // non-negative doubles order like their bit patterns
                    atomicMax(reinterpret_cast<unsigned long long *>(A.partial), (unsigned long long)__double_as_longlong(c));
                    atomicMax(reinterpret_cast<unsigned long long *>(A.partial + 1), (unsigned long long)__double_as_longlong(v));
                }
                cmax = vmax = Real(0);
            }
            if (bad) {
                atomicOr(A.status, DG_STATUS_NONPHYS);
                bad = 0;
            }
        }
        tile = next;
    }
    cp_async_wait_all();
    if (BATCH) return;
    const StageArgs &A = *A0;
    if (bad) s_status = 1;
    if (A.fused) {
        double c = (double)cmax, v = (double)vmax;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            c = fmax(c, __shfl_xor_sync(0xffffffffu, c, off));
            v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
        }
        if ((tid & 31) == 0) {
            s_red[0][tid >> 5] = c;
            s_red[1][tid >> 5] = v;
        }
    }
    __syncthreads();
    if (tid == 0 && s_status) atomicOr(A.status, DG_STATUS_NONPHYS);
    if (A.fused && tid == 0) {
        double c = 0.0, v = 0.0;
        for (int w = 0; w < nth / 32; ++w) {
            c = fmax(c, s_red[0][w]);
            v = fmax(v, s_red[1][w]);
        }
        A.partial[2 * blockIdx.x + 0] = c;
        A.partial[2 * blockIdx.x + 1] = v;
    }
}

template <int DIM, int N, typename Real, bool AV, int NSM, int TX, int TY, int TZ, bool PF>
__global__ void __launch_bounds__(Stage2Plan<DIM, N, Real, AV, NSM, TX, TY, TZ, PF>::NTH,
                                  Stage2Plan<DIM, N, Real, AV, NSM, TX, TY, TZ, PF>::MINB)
    stage2_kernel(const StageArgs A, const Tables<Real> Tg)
{
    stage2_body<DIM, N, Real, AV, NSM, TX, TY, TZ, PF, false>(&A, nullptr, nullptr, 1, Tg);
}

template <int DIM, int N, typename Real, bool AV, int NSM, int TX, int TY, int TZ, bool PF>
__global__ void __launch_bounds__(Stage2Plan<DIM, N, Real, AV, NSM, TX, TY, TZ, PF>::NTH,
                                  Stage2Plan<DIM, N, Real, AV, NSM, TX, TY, TZ, PF>::MINB)
    stage2_batch_kernel(const StageArgs *descs, const int *tile_off, int nsims, const Tables<Real> Tg)
{
    stage2_body<DIM, N, Real, AV, NSM, TX, TY, TZ, PF, true>(nullptr, descs, tile_off, nsims, Tg);
}

template <int DIM, int N, typename Real, bool AV, int NSM, int TX, int TY, int TZ>
constexpr bool stage2_prefetch()
{
    using P1 = Stage2Plan<DIM, N, Real, AV, NSM, TX, TY, TZ, true>;
    using P0 = Stage2Plan<DIM, N, Real, AV, NSM, TX, TY, TZ, false>;
    constexpr size_t sm = 228 * 1024, reserve = 1024;  // shared memory per SM, reserved per CTA
    // 2-D FP32 (two CTAs per SM): the synchronous load fused with pass A measured faster than the
    // prefetch buffers at every degree, one CTA's load overlapping the other's arithmetic
    if (DIM == 2 && sizeof(Real) == 4) return false;
    if (P1::BYTES > 227 * 1024) return false;
    return P1::MINB * (P1::BYTES + reserve) <= sm || P0::MINB * (P0::BYTES + reserve) > sm;
}

template <int DIM, int N, typename Real, bool AV, int NSM, int TX, int TY, int TZ>
cudaError_t run_stage2(const StageArgs &a, const Tables<Real> &t, cudaStream_t s, int *grid_out)
{
    // prefetch buffers (not for 2-D FP32) when the tile still fits in shared memory with them, as
    // many times per SM as the registers are bounded for (else the resident CTAs, not the prefetch,
    // hide latency)
    constexpr bool PF = stage2_prefetch<DIM, N, Real, AV, NSM, TX, TY, TZ>();
    using PL = Stage2Plan<DIM, N, Real, AV, NSM, TX, TY, TZ, PF>;
    auto k = stage2_kernel<DIM, N, Real, AV, NSM, TX, TY, TZ, PF>;
    static_assert(PL::BYTES <= 227 * 1024, "stage2 tile exceeds shared memory");
    static KernelSetup ks;
    int sms = 0, blocks_per_sm = 0;
    cudaError_t e = kernel_setup(ks, k, PL::NTH, PL::BYTES, &sms, &blocks_per_sm);
    if (e != cudaSuccess) return e;
    const int tiles = a.ntile[0] * a.ntile[1] * a.ntile[2];
    if (tiles == 0) return cudaSuccess;
    const int grid = tiles < sms * blocks_per_sm ? tiles : sms * blocks_per_sm;
    if (grid_out) *grid_out = grid;
    k<<<grid, PL::NTH, PL::BYTES, s>>>(a, t);
    return cudaGetLastError();
}

// batched launch: one persistent grid over the (simulation, tile) work list of a group
template <int DIM, int N, typename Real, bool AV, int NSM, int TX, int TY, int TZ>
cudaError_t run_stage2_batch(const StageArgs *descs, const int *tile_off, int nsims, int total_tiles,
                             const Tables<Real> &t, cudaStream_t s)
{
    constexpr bool PF = stage2_prefetch<DIM, N, Real, AV, NSM, TX, TY, TZ>();
    using PL = Stage2Plan<DIM, N, Real, AV, NSM, TX, TY, TZ, PF>;
    auto k = stage2_batch_kernel<DIM, N, Real, AV, NSM, TX, TY, TZ, PF>;
    static KernelSetup ks;  // first call comes from the batch set-up, never from a graph capture
    int sms = 0, blocks_per_sm = 0;
    cudaError_t e = kernel_setup(ks, k, PL::NTH, PL::BYTES, &sms, &blocks_per_sm);
    if (e != cudaSuccess) return e;
    if (total_tiles == 0) return cudaSuccess;
    const int grid = total_tiles < sms * blocks_per_sm ? total_tiles : sms * blocks_per_sm;
    k<<<grid, PL::NTH, PL::BYTES, s>>>(descs, tile_off, nsims, t);
    return cudaGetLastError();
}

template <int DIM, int N, typename Real, int TX, int TY, int TZ>
cudaError_t run_stage2_batch_any(int av, int ns, const StageArgs *descs, const int *tile_off, int nsims,
                                 int total_tiles, const Tables<Real> &t, cudaStream_t s)
{
    if (av) {
        if (ns) return run_stage2_batch<DIM, N, Real, true, 1, TX, TY, TZ>(descs, tile_off, nsims, total_tiles, t, s);
        return run_stage2_batch<DIM, N, Real, true, 0, TX, TY, TZ>(descs, tile_off, nsims, total_tiles, t, s);
    }
    if (ns) return run_stage2_batch<DIM, N, Real, false, 1, TX, TY, TZ>(descs, tile_off, nsims, total_tiles, t, s);
    return run_stage2_batch<DIM, N, Real, false, 0, TX, TY, TZ>(descs, tile_off, nsims, total_tiles, t, s);
}

// run-time (AV, diffusion mode) dispatch onto the compile-time variants.  The tracer plans (TRACER)
// have a tile table of their own (their sixth field takes more shared memory) and always take the
// diffusive path (eta, nu and kappa may be zero); the others are Euler or Navier-Stokes.
template <int DIM, int N, typename Real, int TX, int TY, int TZ, bool TRACER>
cudaError_t run_stage2_any(const StageArgs &a, const Tables<Real> &t, cudaStream_t s, int *grid)
{
    if (!a.tracer_on != !TRACER) return cudaErrorInvalidValue;
    if constexpr (TRACER) {
        if (a.av_on) return run_stage2<DIM, N, Real, true, 2, TX, TY, TZ>(a, t, s, grid);
        return run_stage2<DIM, N, Real, false, 2, TX, TY, TZ>(a, t, s, grid);
    } else {
        if (a.av_on) {
            if (a.ns_on) return run_stage2<DIM, N, Real, true, 1, TX, TY, TZ>(a, t, s, grid);
            return run_stage2<DIM, N, Real, true, 0, TX, TY, TZ>(a, t, s, grid);
        }
        if (a.ns_on) return run_stage2<DIM, N, Real, false, 1, TX, TY, TZ>(a, t, s, grid);
        return run_stage2<DIM, N, Real, false, 0, TX, TY, TZ>(a, t, s, grid);
    }
}

}  // namespace dgx
