// z-marching fused right-hand-side / Runge-Kutta stage kernel for 3-D FP32-bulk grids whose
// degree has Q = n+1 a power of two with Q^2 <= 32 (degrees 1 and 3).
//
// The arithmetic is the collocated rewriting of the modal sums of Eq. time_stepping_final
// (dgx_kernels.cuh, header comment); this file organises it for sm_103a around two facts:
//
//  * a cell's Q^2 x-lines fit in one warp.  Lane group g of a warp owns one cell, lane gl of the
//    group one x-line (y, z) = (gl % Q, gl / Q), held in registers.  Every exchange inside a cell
//    -- the y and z passes of the modal<->nodal transforms, the nodal gradients along y and z and
//    the weak divergence of the y and z fluxes -- is a Q x Q product across the Q lanes that differ
//    in one index, done with xor shuffles, and needs no shared memory and no barrier.  Shared
//    memory holds each cell's nodal values once, for the face phases (lines xor-swizzled so that
//    the strided face-line reads are free of bank conflicts);
//  * a CTA owns a column of TX x TY cells and marches along z through a chunk of planes.  Each
//    plane is loaded and transformed once as the "next" plane, used for the z-faces of the plane
//    below it, and then becomes the current plane; only the x/y face-neighbour ring (2 (TX + TY)
//    cells) is loaded per plane besides.  The flux through the top z-face of a plane is kept and
//    lifted into the plane above at the next step, so every z-face is computed once.
//
// Per plane: (L) load + transform the halo ring of plane z and the own cells of plane z+1;
// (R) recovered interface state of the x/y faces (Navier-Stokes), and the top z-face flux of
// every own cell by the cell's lane group; (F) x/y face fluxes; (V) per own cell and x-line:
// gradients, Euler - NS - AV flux at the line's Q nodes, weak divergence, sources, lifts of the
// six faces, nodal->modal transform and the Runge-Kutta epilogue.  Four block barriers per plane.
// x/y faces on a column boundary are computed by both columns with the same code from the same
// data, so they are bitwise equal on both sides (conservation without atomics).
#pragma once

#include <stdlib.h>

#include "dgx_stage2.cuh"

namespace dgx {

template <int N, bool AV, bool NS, int TX, int TY>
struct Z3Plan {
    static constexpr int Q = N + 1, NP = Q * Q * Q, G = Q * Q;
    static constexpr int NTH = 256, NW = NTH / 32, CPW = 32 / G;
    static constexpr int NC = 5, NF = NC + (AV ? 1 : 0);
    static constexpr int TC = TX * TY, NH = 2 * (TX + TY);
    static_assert((Q & (Q - 1)) == 0 && G <= 32, "lane groups need Q a power of two, Q^2 <= 32");
    static_assert(TC == NW * CPW, "one lane group per own cell of a plane");
    static constexpr int SLOT = NF * NP;  // floats per cell slot: [field][z][y][x]
    static constexpr int NSLOT = 2 * TC + NH;
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1), NFXY = NFX + NFY;
    static constexpr int FH = NC * NFXY * G;            // x/y face fluxes [field][face][point]
    static constexpr int UT = NS ? NC * NFXY * G : 0;   // recovered state at x/y face points
    static constexpr int FZ = 2 * NC * TC * G;          // z-face fluxes [buffer][field][cell][point]
    static constexpr int TAB = 64;                      // lane tables (B, Dn, Wd, G, Lm, Lp)
    static constexpr int OFF_FH = NSLOT * SLOT;
    static constexpr int OFF_UT = OFF_FH + FH;
    static constexpr int OFF_FZ = OFF_UT + UT;
    static constexpr int OFF_WIG = OFF_FZ + FZ;         // [buffer][cell] wiggle source
    static constexpr int OFF_TAB = OFF_WIG + 2 * TC;
    static constexpr int NREAL = OFF_TAB + 6 * TAB;
    static constexpr size_t BYTES = sizeof(float) * (size_t)NREAL + sizeof(int) * (size_t)NSLOT;
    static_assert((OFF_FH * 4) % 16 == 0 && (OFF_UT * 4) % 16 == 0 && (OFF_FZ * 4) % 16 == 0,
                  "vector accesses need 16-byte aligned arrays");
};

// Q x Q matrix-vector product across the Q lanes of a group that differ in one index (the lane's
// index bits selected by STRIDE = 1 (low) or Q (high)): out(i) = sum_j M[i][j] v(j), lane i holding
// v(i).  Recursive doubling: after the first exchange (partner i ^ 1) a lane holds v(i), v(i ^ 1);
// at Q = 4 it then forms the partial sum that its second partner i ^ 2 needs from those two values
// and swaps it, so a product takes log2(Q) shuffles and Q multiply-adds.  The lane's coefficients
// come from xcoef.
template <int Q, int STRIDE>
__device__ __forceinline__ float xmatvec(float v, const float (&Mx)[Q])
{
    static_assert(Q == 2 || Q == 4, "lane products for Q = 2 and 4");
    const float w = __shfl_xor_sync(0xffffffffu, v, STRIDE);
    if constexpr (Q == 2) {
        return fmaf(Mx[1], w, Mx[0] * v);
    } else {
        const float part = fmaf(Mx[3], w, Mx[2] * v);  // M[i^2][i] v(i) + M[i^2][i^1] v(i^1)
        const float recv = __shfl_xor_sync(0xffffffffu, part, 2 * STRIDE);
        return fmaf(Mx[1], w, fmaf(Mx[0], v, recv));
    }
}

// coefficients of lane index i for xmatvec of the Q x Q matrix M (row-major; with T its transpose):
// M[i][i], M[i][i^1] and, at Q = 4, M[i^2][i], M[i^2][i^1]
template <int Q, bool T = false>
__device__ __forceinline__ void xcoef(const float *M, int i, float (&Mx)[Q])
{
    auto e = [&](int r, int c) { return T ? M[c * Q + r] : M[r * Q + c]; };
    Mx[0] = e(i, i);
    Mx[1] = e(i, i ^ 1);
    if constexpr (Q == 4) {
        Mx[2] = e(i ^ 2, i);
        Mx[3] = e(i ^ 2, i ^ 1);
    }
}

// Offset of the x-line (y, z) of one field inside a cell slot.  The Q^2 lines of Q values are
// permuted by an xor swizzle (degree 3: lines with z >= 2 swap y <-> y ^ 2) so that the strided
// reads of the face phases -- the Q lanes of one y-line or z-line position taking the same element
// of different lines -- fall on distinct shared-memory banks; whole-line vector accesses are
// unaffected.
template <int Q>
__device__ __forceinline__ int z3_line(int y, int z)
{
    const int sy = Q == 4 ? (z & 2) : 0;
    return ((y ^ sy) + Q * z) * Q;
}

// the Q values of field f of a cell slot along axis a through the node position (p0, p1) of the
// face numbering (a = 0: x-line at (y, z) = (p0, p1); 1: y-line at (x, z); 2: z-line at (x, y))
template <int Q, int a>
__device__ __forceinline__ void z3_axis_line(const float *slot, int f, int p0, int p1, float (&v)[Q])
{
    constexpr int NP = Q * Q * Q;
    constexpr int VEC = (Q * 4) % 16 == 0 ? 16 : 8;
    const float *b = slot + f * NP;
    if constexpr (a == 0) {
        ld_line<Q, VEC>(b + z3_line<Q>(p0, p1), v);
    } else if constexpr (a == 1) {
#pragma unroll
        for (int m = 0; m < Q; ++m) v[m] = b[z3_line<Q>(m, p1) + p0];
    } else {
#pragma unroll
        for (int m = 0; m < Q; ++m) v[m] = b[z3_line<Q>(p1, m) + p0];
    }
}

// recovered state at one face point (Sec. 3.2): q = sum_m Cm[m] left line + Cp[m] right line
template <int Q, int a>
__device__ __forceinline__ void z3_recover(const float *sl, const float *sr, int p0, int p1, const Tables<float> &Tg,
                                           float (&ut)[5])
{
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        float lv[Q], rv[Q];
        z3_axis_line<Q, a>(sl, f, p0, p1, lv);
        z3_axis_line<Q, a>(sr, f, p0, p1, rv);
        float acc = 0.0f;
#pragma unroll
        for (int m = 0; m < Q; ++m) acc = fmaf(Tg.Cm[m], lv[m], fmaf(Tg.Cp[m], rv[m], acc));
        ut[f] = acc;
    }
}

// flux through one face point normal to axis a, before weighting: HLLC of the two traces minus the
// Navier-Stokes flux of the recovered state ut with tangential derivatives gtan and the recovered
// normal derivative, minus the artificial-viscosity flux eps_face d_n u.  Either side may be absent
// (outflow boundary: sl or sr null): then the physical flux of the interior trace, no dissipation.
template <int Q, bool AV, bool NS, int a>
__device__ __forceinline__ void z3_face_flux(const float *sl, const float *sr, int p0, int p1, const float (&ut)[5],
                                             const float (&gtan)[3][5], const Tables<float> &Tg, const StageArgs &A,
                                             float (&Fh)[5], int &bad)
{
    constexpr int NC = 5, NF = NC + (AV ? 1 : 0);
    constexpr bool GRAD = AV || NS;
    if (!sl || !sr) {
        const float *si = sl ? sl : sr;
        float u[NF], v[3], rho, pr_, cs;
#pragma unroll
        for (int f = 0; f < NC; ++f) {
            float q[Q];
            z3_axis_line<Q, a>(si, f, p0, p1, q);
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m < Q; ++m) acc = fmaf(sl ? Tg.Lp[m] : Tg.Lm[m], q[m], acc);
            u[f] = acc;
        }
        if (!primitives<3>(u, A.kf[SK_GAMMA], rho, v, pr_, cs)) bad = 1;
        euler_flux<3, false>(u, v, pr_, a, Fh);
        return;
    }
    float uL[NC + 1], uR[NC + 1], dn[NC];
    const float sc = Tg.inv_f * A.kf[SK_INV_H + a];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        float lv[Q], rv[Q];
        z3_axis_line<Q, a>(sl, f, p0, p1, lv);
        z3_axis_line<Q, a>(sr, f, p0, p1, rv);
        float al = 0.0f, ar = 0.0f;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            al = fmaf(Tg.Lp[m], lv[m], al);
            ar = fmaf(Tg.Lm[m], rv[m], ar);
        }
        uL[f] = al;
        uR[f] = ar;
        if (GRAD && f < NC) {
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m < Q; ++m) acc = fmaf(Tg.Dm[m], lv[m], fmaf(Tg.Dp[m], rv[m], acc));
            dn[f] = acc * sc;
        }
    }
    float cL, cR;
    if (!hllc<3, false>(uL, uR, A.kf[SK_GAMMA], a, Fh, cL, cR)) bad = 1;
    if constexpr (NS) {
        float grd[3][NC];
#pragma unroll
        for (int f = 0; f < NC; ++f) {
#pragma unroll
            for (int b = 0; b < 3; ++b) grd[b][f] = b == a ? dn[f] : gtan[b][f];
        }
        if (!(ut[0] > 0.0f)) bad = 1;
        float Fn[NC];
        ns_flux<3, false>(ut, grd, A.kf[SK_GAMMA], A.kf[SK_NU], A.kf[SK_KAPPA], 0.0f, a, Fn);
#pragma unroll
        for (int f = 0; f < NC; ++f) Fh[f] -= Fn[f];
    }
    if constexpr (AV) {
        const float eps = 0.5f * A.kf[SK_EPS] * (clamp01(uL[NC]) * cL + clamp01(uR[NC]) * cR);
#pragma unroll
        for (int f = 0; f < NC; ++f) Fh[f] -= eps * dn[f];
    }
}

// flux of one x- (a = 0) or y- (a = 1) face point, weighted for the lift, into sFh; with NS the
// recovered state and its tangential derivatives come from sUt (face numbering (p0, p1))
template <int Q, bool AV, bool NS, int NFXY, int a>
__device__ __forceinline__ void z3_xy_flux(const float *sl, const float *sr, int face, int p0, int p1, int k,
                                           const float *sUt, const float *tDn, const float *tG,
                                           const Tables<float> &Tg, const StageArgs &A, float *sFh, int &bad)
{
    constexpr int NC = 5, G = Q * Q;
    constexpr int ta = a == 0 ? 1 : 0;  // first tangential axis (p0); the second is z (p1)
    float ut[NC], gtan[3][NC];
    if (NS && sl && sr) {
        const float *pf = sUt + face * G;
#pragma unroll
        for (int f = 0; f < NC; ++f) {
            const float *pp = pf + f * NFXY * G;
            ut[f] = pp[p0 + Q * p1];
            float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                a0 = fmaf(tDn[p0 * Q + m], pp[m + Q * p1], a0);
                a1 = fmaf(tDn[p1 * Q + m], pp[p0 + Q * m], a1);
            }
            gtan[a][f] = 0.0f;
            gtan[ta][f] = a0 * A.kf[SK_TWO_H + ta];
            gtan[2][f] = a1 * A.kf[SK_TWO_H + 2];
        }
    }
    float Fh[NC];
    z3_face_flux<Q, AV, NS, a>(sl, sr, p0, p1, ut, gtan, Tg, A, Fh, bad);
    const float w = A.kf[SK_CAX + a] * tG[p0] * tG[p1];
#pragma unroll
    for (int f = 0; f < NC; ++f) sFh[(f * NFXY + face) * G + k] = w * Fh[f];
}

// One modal x-line of a global state array: Q values with the widest aligned vector accesses, or, in
// packed total-degree storage, the line's len stored modes (scalar; the others read as zero, are not
// written)
template <int Q, int VEC, typename T>
__device__ __forceinline__ void z3_ld(const T *p, bool packed, int len, T (&w)[Q])
{
    if (!packed) {  // (packed is a compile-time constant at every call)
        ld_line<Q, VEC>(p, w);
        return;
    }
#pragma unroll
    for (int m = 0; m < Q; ++m) w[m] = m < len ? p[m] : T(0);
}
template <int Q, int VEC, typename T>
__device__ __forceinline__ void z3_st(T *p, bool packed, int len, const T (&w)[Q])
{
    if (!packed) {
        st_line<Q, VEC>(p, w);
        return;
    }
#pragma unroll
    for (int m = 0; m < Q; ++m)
        if (m < len) p[m] = w[m];
}

template <int N, bool AV, bool NS, int TX, int TY, bool PK>
__global__ void __launch_bounds__(256, 2) stage3z_kernel(const StageArgs A, const Tables<float> Tg)
{
    using PL = Z3Plan<N, AV, NS, TX, TY>;
    constexpr int Q = PL::Q, NP = PL::NP, G = PL::G, NC = PL::NC, NF = PL::NF, TC = PL::TC, NH = PL::NH;
    constexpr int NFX = PL::NFX, NFXY = PL::NFXY, NTH = PL::NTH;
    constexpr int VEC = (Q * 4) % 16 == 0 ? 16 : 8;
    constexpr bool GRAD = AV || NS;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    float *sFh = sm + PL::OFF_FH, *sUt = sm + PL::OFF_UT, *sFz = sm + PL::OFF_FZ, *sWig = sm + PL::OFF_WIG;
    float *tB = sm + PL::OFF_TAB, *tDn = tB + PL::TAB, *tWd = tDn + PL::TAB, *tG = tWd + PL::TAB;
    float *tLm = tG + PL::TAB, *tLp = tLm + PL::TAB;
    int *sG = reinterpret_cast<int *>(sm + PL::NREAL);
    __shared__ double s_red[2][NTH / 32];
    __shared__ double s_dt;
    __shared__ int s_status;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gl = lane % G;              // x-line of the lane within its cell: (y, z) = (gl % Q, gl / Q)
    const int grp = warp * PL::CPW + lane / G;  // own-cell index of the lane group within a plane
    const int ly = gl % Q, lz = gl / Q;

    for (int i = tid; i < Q * Q; i += NTH) {
        tB[i] = Tg.B[i / Q][i % Q];
        tDn[i] = Tg.Dn[i / Q][i % Q];
        tWd[i] = Tg.Wd[i / Q][i % Q];
    }
    for (int i = tid; i < Q; i += NTH) {
        tG[i] = Tg.G[i];
        tLm[i] = Tg.Lm[i];
        tLp[i] = Tg.Lp[i];
    }
    if (tid == 0) s_status = 0;

    // time step of the step from the first stage's per-CTA maxima (Eq. timestep), identical in every CTA
    if (A.dt_partial) {
        double c = 0.0, v = 0.0;
        for (int i = tid; i < A.dt_nblk; i += NTH) {
            c = fmax(c, A.dt_partial[2 * i]);
            v = fmax(v, A.dt_partial[2 * i + 1]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            c = fmax(c, __shfl_xor_sync(0xffffffffu, c, off));
            v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
        }
        if (lane == 0) {
            s_red[0][warp] = c;
            s_red[1][warp] = v;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < NTH / 32; ++w) {
                c = fmax(c, s_red[0][w]);
                v = fmax(v, s_red[1][w]);
            }
            const double dt = A.dt_fixed > 0.0 ? A.dt_fixed : A.cfl * A.hmin / (2.0 * (N + 1) * (c + v));
            s_dt = dt;
            if (blockIdx.x == 0) {
                if (!(dt > 0.0) || !isfinite(dt)) atomicOr(A.status, DG_STATUS_BADDT);
                double *dtp = const_cast<double *>(A.dtp);
                dtp[0] = dt;
                dtp[1] += 1.0;
                dtp[2] += dt;
            }
        }
    }
    __syncthreads();

    // per-simulation constants: read from the kernel parameter (A.kf) where used
    const float *K = A.kf;
    const double dstep = A.dt_partial ? s_dt : (A.dtp ? A.dtp[0] : 0.0);
    const float dt = A.epi_unit_dt ? 1.0f : (A.mode != 0 ? (float)dstep : 0.0f);
    const float dsc = A.din_dt ? (float)(A.din_coef * dstep) : 1.0f;
    const float ca = K[SK_CA], cxc = K[SK_CX], cb = K[SK_CB];
    const float za = K[SK_ZA], zx = K[SK_ZX], zb = K[SK_ZB];
    const float *ub = static_cast<const float *>(A.ubase);
    const float *di = static_cast<const float *>(A.din);
    float *xb = static_cast<float *>(A.xbuf);
    float *dout = static_cast<float *>(A.dout);
    const bool readx = xb && (A.cx != 0.0 || A.zx != 0.0);
    const int N0 = A.N[0], N1 = A.N[1], N2 = A.N[2];
    // stored modes per cell, and the lane's modal x-line (l_y, l_z) = (ly, lz) in the global arrays:
    // tensor storage, or packed total-degree storage (the line's modes l_x <= n - l_y - l_z)
    constexpr bool packed = PK;  // PK: packed total-degree storage (a separate instantiation)
    const int MS = packed ? A.ms : NP;
    const int plen = packed ? max(0, N + 1 - ly - lz) : Q;
    const int poff = packed ? (plen > 0 ? A.cmap[Q * (ly + Q * lz)] : 0) : gl * Q;
    const size_t fstride = (size_t)A.ncell * MS;  // values between fields

    float cmax = 0.0f, vmax = 0.0f;  // CFL speeds (fused first stage)
    int bad = 0;

    // global cell index of tile position (cx, cy) in plane z (-1: outside the domain with an outflow
    // boundary); positions run one beyond the tile on each side (the face-neighbour ring)
    auto gcell = [&](int o0, int o1, int cx, int cy, int z) -> int {
        int gx = o0 + cx, gy = o1 + cy;
        if (gx < 0 || gx >= N0) {
            if (A.bc[0] != 0) return -1;
            gx = (gx + N0) % N0;
        }
        if (gy < 0 || gy >= N1) {
            if (A.bc[1] != 0) return -1;
            gy = (gy + N1) % N1;
        }
        return gx + N0 * (gy + N1 * z);
    };
    // plane index of z + dz, or -1 beyond an outflow boundary
    auto zplane = [&](int z) -> int {
        if (z < 0 || z >= N2) {
            if (A.bc[2] != 0) return -1;
            return (z + N2) % N2;
        }
        return z;
    };

    // (L) one cell by one lane group: u^n (+ delta) x-line of every field, modal -> nodal along x in
    // registers, then y and z through the cell's slot; with `sensor`, the oscillation sensor of the
    // modal density and the wiggle source of Sec. 4.1 (fused first stage), stored to *wig_slot
    auto load_cell = [&](float *slot, int g, bool sensor, float *wig_slot) {
        const bool valid = g >= 0;
        float w[NF][Q];
        if (valid) {
            const size_t g0 = (size_t)g * MS + (size_t)poff;
#pragma unroll
            for (int f = 0; f < NF; ++f) z3_ld<Q, VEC>(ub + g0 + f * fstride, packed, plen, w[f]);
            if (di) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    float dd[Q];
                    z3_ld<Q, VEC>(di + g0 + f * fstride, packed, plen, dd);
#pragma unroll
                    for (int m = 0; m < Q; ++m) w[f][m] = w[f][m] + dsc * dd[m];
                }
            }
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int m = 0; m < Q; ++m) w[f][m] = 0.0f;
        }
        if (AV && sensor) {
            // sum of squares of the density modes, all and those the degree-(n-1) basis lacks
            float all = 0.0f, hi = 0.0f;
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                const bool top = A.total_degree ? (m + ly + lz == N) : (m == N || ly == N || lz == N);
                all += w[0][m] * w[0][m];
                if (top) hi += w[0][m] * w[0][m];
            }
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                all += __shfl_xor_sync(0xffffffffu, all, off);
                hi += __shfl_xor_sync(0xffffffffu, hi, off);
            }
            if (valid && gl == 0) {
                const double Sk = all > 0.0f ? (double)(hi / all) : 0.0;
                const double dt_prev = A.dtp[0], step = A.dtp[1];
                const float sf = (float)(1e-4 * A.s_on);
                double dlog = 0.0;
                if (step > 0.0 && dt_prev > 0.0)
                    dlog = (double)((logf(fmaxf((float)Sk, sf)) - logf(fmaxf((float)A.S_prev[g], sf))) /
                                    (float)dt_prev);
                const double wg = (Sk > A.s_on) ? A.f_w * fmax(0.0, dlog) : 0.0;
                A.wig_w[g] = wg;
                A.S_prev[g] = Sk;
                *wig_slot = (float)wg;
            }
        } else if (AV && valid && gl == 0 && wig_slot) {
            *wig_slot = (float)A.wig[g];
        }
        // x: modal -> nodal in registers
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            float o[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float acc = 0.0f;
#pragma unroll
                for (int m = 0; m < Q; ++m) acc = fmaf(Tg.B[i][m], w[f][m], acc);
                o[i] = acc;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) w[f][i] = o[i];
        }
        // y then z across the group's lanes (xor shuffles): out(i) = sum_m B[i][m] v(m), the lane of
        // index i holding v(i)
        float by[Q], bz[Q];
        xcoef<Q>(tB, ly, by);
        xcoef<Q>(tB, lz, bz);
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int i = 0; i < Q; ++i) w[f][i] = xmatvec<Q, 1>(w[f][i], by);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
#pragma unroll
            for (int i = 0; i < Q; ++i) w[f][i] = xmatvec<Q, Q>(w[f][i], bz);
            st_line<Q, VEC>(slot + f * NP + z3_line<Q>(ly, lz), w[f]);
        }
    };

    // z-face between the lane group's cell in slot sl (below) and slot sr (above), at the face point
    // (x, y) = (gl % Q, gl / Q), by all lanes of the group; the weighted flux goes to fz[f * TC * G + gl]
    auto zface = [&](const float *sl, const float *sr, bool valid, float *fz) {
        const int px = gl % Q, py = gl / Q;
        float ut[NC];
        float gtan[3][NC];
        if (NS) {
            if (sl && sr) z3_recover<Q, 2>(sl, sr, px, py, Tg, ut);
            else {
#pragma unroll
                for (int f = 0; f < NC; ++f) ut[f] = 0.0f;
            }
            // tangential derivatives of the recovered state: across the group's lanes (all lanes take part)
            float dx[Q], dy[Q];
            xcoef<Q>(tDn, px, dx);
            xcoef<Q>(tDn, py, dy);
#pragma unroll
            for (int f = 0; f < NC; ++f) {
                gtan[0][f] = xmatvec<Q, 1>(ut[f], dx) * K[SK_TWO_H + 0];
                gtan[1][f] = xmatvec<Q, Q>(ut[f], dy) * K[SK_TWO_H + 1];
                gtan[2][f] = 0.0f;
            }
        }
        if (!valid) return;
        float Fh[NC];
        z3_face_flux<Q, AV, NS, 2>(sl, sr, px, py, ut, gtan, Tg, A, Fh, bad);
        const float w = K[SK_CAX + 2] * tG[px] * tG[py];
#pragma unroll
        for (int f = 0; f < NC; ++f) fz[f * TC * G + gl] = w * Fh[f];
    };

    // work items: (column, z-chunk); the chunk length comes with the arguments
    const int ntx = A.ntile[0], nty = A.ntile[1], nzc = A.ntile[2];
    const int ZC = A.zchunk;
    const int nitems = ntx * nty * nzc;
    // own-cell buffers b = 0, 1 of planes (slots b TC + c) and their global cells; the halo ring
    auto own = [&](int b) { return sm + b * TC * PL::SLOT; };
    auto gOwn = [&](int b) { return sG + b * TC; };
    float *halo = sm + 2 * TC * PL::SLOT;
    int *gHalo = sG + 2 * TC;

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        int b = item;
        const int tx = b % ntx;
        b /= ntx;
        const int ty = b % nty;
        const int zc = b / nty;
        const int o0 = tx * TX, o1 = ty * TY;
        const int V0 = min(TX, N0 - o0), V1 = min(TY, N1 - o1);
        const int z0 = zc * ZC, z1 = min(N2, z0 + ZC);
        int cur = 0;  // own buffer of the current plane
        const int mcx = grp % TX, mcy = grp / TX;
        const bool mine = mcx < V0 && mcy < V1;

        // chunk prologue: plane z0 - 1 into buffer 1, plane z0 into buffer 0 (with the sensor), the
        // z-faces between them -> bottom-face fluxes of plane z0 (buffer 1 of sFz)
        {
            const int zp = zplane(z0 - 1);
            if (tid < TC) {
                const int cx = tid % TX, cy = tid / TX;
                const bool in = cx < V0 && cy < V1;
                gOwn(0)[tid] = in ? gcell(o0, o1, cx, cy, z0) : -1;
                gOwn(1)[tid] = (in && zp >= 0) ? gcell(o0, o1, cx, cy, zp) : -1;
            }
            __syncthreads();
            load_cell(own(0) + grp * PL::SLOT, gOwn(0)[grp], A.fused != 0, sWig + grp);
            load_cell(own(1) + grp * PL::SLOT, gOwn(1)[grp], false, nullptr);
            __syncthreads();
            const bool below = zp >= 0;
            zface(below ? own(1) + grp * PL::SLOT : nullptr, own(0) + grp * PL::SLOT, mine,
                  sFz + NC * TC * G + grp * G);
            __syncthreads();
        }

        for (int z = z0; z < z1; ++z) {
            const int nxt = 1 - cur;
            const int zn = zplane(z + 1);
            float *sCur = own(cur), *sNxt = own(nxt);
            // (L) slot maps, then the halo ring of plane z and the own cells of plane z + 1
            if (tid < NH) {
                const int h = tid;
                int cx, cy;
                bool in;
                if (h < TY) {
                    cx = -1;
                    cy = h;
                    in = cy < V1;
                } else if (h < 2 * TY) {
                    cx = V0;
                    cy = h - TY;
                    in = cy < V1;
                } else if (h < 2 * TY + TX) {
                    cx = h - 2 * TY;
                    cy = -1;
                    in = cx < V0;
                } else {
                    cx = h - 2 * TY - TX;
                    cy = V1;
                    in = cx < V0;
                }
                gHalo[h] = in ? gcell(o0, o1, cx, cy, z) : -1;
            } else if (tid >= 32 && tid < 32 + TC) {
                const int c = tid - 32;
                const int cx = c % TX, cy = c / TX;
                gOwn(nxt)[c] = (cx < V0 && cy < V1 && zn >= 0) ? gcell(o0, o1, cx, cy, zn) : -1;
            }
            __syncthreads();
            // the next plane's sensor and wiggle source belong to this chunk unless the next plane
            // starts another chunk (whose prologue computes them)
            const bool nown = z + 1 < z1;
            const bool nsens = A.fused != 0 && nown;
            for (int t = grp; t < NH + TC; t += TC) {
                if (t < NH) load_cell(halo + t * PL::SLOT, gHalo[t], false, nullptr);
                else load_cell(sNxt + (t - NH) * PL::SLOT, gOwn(nxt)[t - NH], nsens,
                               nown ? sWig + nxt * TC + (t - NH) : nullptr);
            }
            __syncthreads();

            // slot of tile position (cx, cy) of plane z for the face phases (halo positions included)
            auto slot_at = [&](int cx, int cy) -> const float * {
                int s = -1;
                if (cx >= 0 && cx < V0 && cy >= 0 && cy < V1) return sCur + (cx + TX * cy) * PL::SLOT;
                if (cx == -1) s = cy;
                else if (cx == V0) s = TY + cy;
                else if (cy == -1) s = 2 * TY + cx;
                else s = 2 * TY + TX + cx;
                return gHalo[s] >= 0 ? halo + s * PL::SLOT : nullptr;
            };
            // decode x/y face point q: axis, the two sides, face index and point (p0, p1) in the face
            auto face_of = [&](int q, int &a, const float *&sl, const float *&sr, int &face, int &p0, int &p1) -> bool {
                face = q / G;
                const int k = q % G;
                p0 = k % Q;
                p1 = k / Q;
                if (face < NFX) {
                    a = 0;
                    const int px = face % (TX + 1), cy = face / (TX + 1);
                    if (px > V0 || cy >= V1) return false;
                    sl = slot_at(px - 1, cy);
                    sr = slot_at(px, cy);
                } else {
                    a = 1;
                    const int fy = face - NFX;
                    const int cx = fy % TX, py = fy / TX;
                    if (cx >= V0 || py > V1) return false;
                    sl = slot_at(cx, py - 1);
                    sr = slot_at(cx, py);
                }
                return sl || sr;
            };

            // (R) recovered state at the x/y face points; the top z-face of every own cell
            if (NS) {
                for (int q = tid; q < NFXY * G; q += NTH) {
                    int a, face, p0, p1;
                    const float *sl, *sr;
                    if (!face_of(q, a, sl, sr, face, p0, p1) || !sl || !sr) continue;
                    float ut[NC];
                    if (a == 0) z3_recover<Q, 0>(sl, sr, p0, p1, Tg, ut);
                    else z3_recover<Q, 1>(sl, sr, p0, p1, Tg, ut);
#pragma unroll
                    for (int f = 0; f < NC; ++f) sUt[(f * NFXY + face) * G + q % G] = ut[f];
                }
            }
            zface(sCur + grp * PL::SLOT, zn >= 0 ? sNxt + grp * PL::SLOT : nullptr, mine,
                  sFz + cur * NC * TC * G + grp * G);
            __syncthreads();

            // (F) x/y face fluxes, weighted for the lift (one code path per axis, the axis a
            // compile-time constant)
            for (int q = tid; q < NFXY * G; q += NTH) {
                int a, face, p0, p1;
                const float *sl, *sr;
                if (!face_of(q, a, sl, sr, face, p0, p1)) continue;
                if (a == 0)
                    z3_xy_flux<Q, AV, NS, NFXY, 0>(sl, sr, face, p0, p1, q % G, sUt, tDn, tG, Tg, A, sFh, bad);
                else
                    z3_xy_flux<Q, AV, NS, NFXY, 1>(sl, sr, face, p0, p1, q % G, sUt, tDn, tG, Tg, A, sFh, bad);
            }
            __syncthreads();

            // (V) own cells: volume terms, sources and lifts on the lane's x-line, then the transposed
            // transform and the Runge-Kutta epilogue
            {
                float *slot = sCur + grp * PL::SLOT;
                const int g = gOwn(cur)[grp];
                float u[NF][Q];
#pragma unroll
                for (int f = 0; f < NF; ++f) ld_line<Q, VEC>(slot + f * NP + z3_line<Q>(ly, lz), u[f]);
                float dy[Q], dz[Q], wy[Q], wz[Q];
                xcoef<Q>(tDn, ly, dy);
                xcoef<Q>(tDn, lz, dz);
                xcoef<Q>(tWd, ly, wy);
                xcoef<Q>(tWd, lz, wz);
                const float gy = tG[ly], gz = tG[lz];
                const float wig = AV ? sWig[cur * TC + grp] : 0.0f;
                const float *force = static_cast<const float *>(A.force);
                float r[NF][Q];
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int i = 0; i < Q; ++i) r[f][i] = 0.0f;
#pragma unroll
                for (int x = 0; x < Q; ++x) {
                    float uu[NC + 1];
#pragma unroll
                    for (int f = 0; f < NF; ++f) uu[f] = u[f][x];
                    float gr[3][NC];
                    if (GRAD) {
#pragma unroll
                        for (int f = 0; f < NC; ++f) {
                            float acc = 0.0f;
#pragma unroll
                            for (int m = 0; m < Q; ++m) acc = fmaf(Tg.Dn[x][m], u[f][m], acc);
                            gr[0][f] = acc * K[SK_TWO_H + 0];
                            gr[1][f] = xmatvec<Q, 1>(u[f][x], dy) * K[SK_TWO_H + 1];
                            gr[2][f] = xmatvec<Q, Q>(u[f][x], dz) * K[SK_TWO_H + 2];
                        }
                    }
                    float rho, v[3], p, cs;
                    if (!primitives<3>(uu, K[SK_GAMMA], rho, v, p, cs) && mine) bad = 1;
                    if (A.fused && mine) {
                        cmax = fmaxf(cmax, cs);
                        vmax = fmaxf(vmax, sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
                    }
                    const float eps = AV ? K[SK_EPS] * clamp01(uu[NC]) * cs : 0.0f;
                    float Fns[3][NC];
                    if (NS) ns_flux_all<3>(uu, gr, K[SK_GAMMA], K[SK_NU], K[SK_KAPPA], Fns);
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        float F[NC];
                        euler_flux<3, false>(uu, v, p, a, F);
                        if (NS) {
#pragma unroll
                            for (int f = 0; f < NC; ++f) F[f] -= Fns[a][f];
                        }
                        if (AV) {
#pragma unroll
                            for (int f = 0; f < NC; ++f) F[f] -= eps * gr[a][f];
                        }
                        if (a == 0) {
                            const float w = K[SK_CAX + 0] * gy * gz;
#pragma unroll
                            for (int f = 0; f < NC; ++f)
#pragma unroll
                                for (int i = 0; i < Q; ++i) r[f][i] = fmaf(Tg.Wd[i][x] * w, F[f], r[f][i]);
                        } else if (a == 1) {
                            const float w = K[SK_CAX + 1] * Tg.G[x] * gz;
#pragma unroll
                            for (int f = 0; f < NC; ++f) r[f][x] += xmatvec<Q, 1>(w * F[f], wy);
                        } else {
                            const float w = K[SK_CAX + 2] * Tg.G[x] * gy;
#pragma unroll
                            for (int f = 0; f < NC; ++f) r[f][x] += xmatvec<Q, Q>(w * F[f], wz);
                        }
                    }
                    const float Gv = Tg.G[x] * gy * gz;
                    if (force && mine) {
                        // driving source of Sec. 7.1: rho s into the momentum, s.(rho v) into the energy
                        const float wgt = 0.125f * Gv;
                        float se = 0.0f;
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float sa = force[((size_t)a * A.ncell + g) * NP + gl * Q + x];
                            r[1 + a][x] = fmaf(wgt * uu[0], sa, r[1 + a][x]);
                            se = fmaf(sa, uu[1 + a], se);
                        }
                        r[4][x] = fmaf(wgt, se, r[4][x]);
                    }
                    if (AV) {
                        float div = 0.0f;
#pragma unroll
                        for (int a = 0; a < 3; ++a) div += (gr[a][1 + a] - v[a] * gr[a][0]) / rho;
                        const float adot = K[SK_FV] * fmaxf(0.0f, -div) + wig - uu[NC] * cs * K[SK_INV_TAU];
                        r[NC][x] = 0.125f * Gv * adot;
                    }
                }
                // lifts of the six face fluxes
                {
                    const int fxl = mcx + (TX + 1) * mcy;            // x-faces left / right: points (y, z)
                    const int fyb = NFX + mcx + TX * mcy;            // y-faces bottom / top: points (x, z)
                    const float lmy = tLm[ly], lpy = tLp[ly], lmz = tLm[lz], lpz = tLp[lz];
                    const float *fzb = sFz + (1 - cur) * NC * TC * G + grp * G;  // bottom: last plane's top
                    const float *fzt = sFz + cur * NC * TC * G + grp * G;
#pragma unroll
                    for (int f = 0; f < NC; ++f) {
                        if (mine) {
                            const float fL = sFh[(f * NFXY + fxl) * G + gl];
                            const float fR = sFh[(f * NFXY + fxl + 1) * G + gl];
                            float yb[Q], yt[Q], zb_[Q], zt[Q];
                            ld_line<Q, VEC>(sFh + (f * NFXY + fyb) * G + Q * lz, yb);
                            ld_line<Q, VEC>(sFh + (f * NFXY + fyb + TX) * G + Q * lz, yt);
                            ld_line<Q, VEC>(fzb + f * TC * G + Q * ly, zb_);
                            ld_line<Q, VEC>(fzt + f * TC * G + Q * ly, zt);
#pragma unroll
                            for (int i = 0; i < Q; ++i) {
                                float acc = r[f][i];
                                acc = fmaf(Tg.Lm[i], fL, acc);
                                acc = fmaf(-Tg.Lp[i], fR, acc);
                                acc = fmaf(lmy, yb[i], acc);
                                acc = fmaf(-lpy, yt[i], acc);
                                acc = fmaf(lmz, zb_[i], acc);
                                r[f][i] = fmaf(-lpz, zt[i], acc);
                            }
                        }
                    }
                }
                // nodal -> modal: z then y across the group's lanes, out(l) = sum_i B[i][l] r(i); x in registers
                float cz_[Q], cy_[Q];
                xcoef<Q, true>(tB, lz, cz_);
                xcoef<Q, true>(tB, ly, cy_);
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int i = 0; i < Q; ++i) r[f][i] = xmatvec<Q, 1>(xmatvec<Q, Q>(r[f][i], cz_), cy_);
                if (mine) {
                    // epilogue on the modal x-line (l_y, l_z) = (ly, lz)
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const size_t gi = (size_t)f * fstride + (size_t)g * MS + (size_t)poff;
                        constexpr int VD = (Q * 8) % 16 == 0 ? 16 : 8;
                        double uo[Q];
                        if (A.mode == 2) z3_ld<Q, VD>(A.uold + gi, packed, plen, uo);
                        float L[Q];
#pragma unroll
                        for (int l = 0; l < Q; ++l) {
                            float acc = 0.0f;
#pragma unroll
                            for (int i = 0; i < Q; ++i) acc = fmaf(Tg.B[i][l], r[f][i], acc);
                            L[l] = acc;
                        }
                        if (A.total_degree) {
#pragma unroll
                            for (int l = 0; l < Q; ++l)
                                if (l + ly + lz > N) L[l] = 0.0f;
                        }
                        if (A.mode == 0) {
#pragma unroll
                            for (int l = 0; l < Q; ++l)
                                if (l < plen) A.rhs_out[gi + l] = (double)L[l];
                            continue;
                        }
                        float din[Q], xv[Q], dnew[Q], zn_[Q];
                        if (di) {
                            z3_ld<Q, VEC>(di + gi, packed, plen, din);
#pragma unroll
                            for (int l = 0; l < Q; ++l) din[l] = dsc * din[l];
                        } else {
#pragma unroll
                            for (int l = 0; l < Q; ++l) din[l] = 0.0f;
                        }
                        if (readx) {
                            z3_ld<Q, VEC>(xb + gi, packed, plen, xv);
                        } else {
#pragma unroll
                            for (int l = 0; l < Q; ++l) xv[l] = 0.0f;
                        }
#pragma unroll
                        for (int l = 0; l < Q; ++l) {
                            const float dtL = dt * L[l];
                            dnew[l] = ca * din[l] + cxc * xv[l] + cb * dtL;
                            zn_[l] = za * din[l] + zx * xv[l] + zb * dtL;
                        }
                        if (A.write_z) z3_st<Q, VEC>(xb + gi, packed, plen, zn_);
                        if (A.mode == 1) {
                            z3_st<Q, VEC>(dout + gi, packed, plen, dnew);
                        } else {
                            double un[Q];
#pragma unroll
                            for (int l = 0; l < Q; ++l) un[l] = uo[l] + (double)dnew[l];
                            z3_st<Q, VD>(A.unew + gi, packed, plen, un);
                            if (A.uhi_new) {
                                float uf[Q];
#pragma unroll
                                for (int l = 0; l < Q; ++l) uf[l] = (float)un[l];
                                z3_st<Q, VEC>(A.uhi_new + gi, packed, plen, uf);
                            }
                        }
                    }
                }
            }
            cur = nxt;
            __syncthreads();
        }
    }

    if (bad) s_status = 1;
    if (A.fused) {
        double c = (double)cmax, v = (double)vmax;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            c = fmax(c, __shfl_xor_sync(0xffffffffu, c, off));
            v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
        }
        if (lane == 0) {
            s_red[0][warp] = c;
            s_red[1][warp] = v;
        }
    }
    __syncthreads();
    if (tid == 0 && s_status) atomicOr(A.status, DG_STATUS_NONPHYS);
    if (A.fused && tid == 0) {
        double c = 0.0, v = 0.0;
        for (int w = 0; w < NTH / 32; ++w) {
            c = fmax(c, s_red[0][w]);
            v = fmax(v, s_red[1][w]);
        }
        A.partial[2 * blockIdx.x + 0] = c;
        A.partial[2 * blockIdx.x + 1] = v;
    }
}

// chunking of the z-march: the chunk length that minimises the planes the busiest CTA processes
// (rounds of (column, chunk) items over the resident CTAs, times the chunk length plus the plane
// below it that every chunk loads again)
inline void z3_items(int ntx, int nty, int N2, int ctas, int *nzc, int *zchunk)
{
    long long best = -1;
    for (int c = 1; c <= N2; ++c) {
        const int zc = (N2 + c - 1) / c;
        const int n = (N2 + zc - 1) / zc;
        const long long items = (long long)ntx * nty * n;
        const long long rounds = (items + ctas - 1) / ctas;
        const long long cost = rounds * (zc + 1);
        if (best < 0 || cost < best) {
            best = cost;
            *zchunk = zc;
            *nzc = n;
        }
    }
}

template <int N, bool AV, bool NS, int TX, int TY, bool PK>
cudaError_t run_stage3z(const StageArgs &a_in, const Tables<float> &t, cudaStream_t s, int *grid_out)
{
    using PL = Z3Plan<N, AV, NS, TX, TY>;
    auto k = stage3z_kernel<N, AV, NS, TX, TY, PK>;
    static_assert(PL::BYTES <= 227 * 1024, "z-march plane exceeds shared memory");
    static KernelSetup ks;
    int sms = 0, per_sm = 0;
    cudaError_t e = kernel_setup(ks, k, PL::NTH, PL::BYTES, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    StageArgs a = a_in;
    a.ntile[0] = (a.N[0] + TX - 1) / TX;
    a.ntile[1] = (a.N[1] + TY - 1) / TY;
    const int ctas = sms * per_sm;
    z3_items(a.ntile[0], a.ntile[1], a.N[2], ctas, &a.ntile[2], &a.zchunk);
    // DGX_ZCHUNK=k: k planes per chunk instead of the automatic choice (a tuning and test knob; the
    // arithmetic does not depend on it)
    if (const char *zc = getenv("DGX_ZCHUNK")) {
        const int k = atoi(zc);
        if (k > 0) {
            a.zchunk = k < a.N[2] ? k : a.N[2];
            a.ntile[2] = (a.N[2] + a.zchunk - 1) / a.zchunk;
        }
    }
    if (a_in.ntile[0] * a_in.ntile[1] * a_in.ntile[2] == 0) return cudaSuccess;  // set-up call
    const int items = a.ntile[0] * a.ntile[1] * a.ntile[2];
    const int grid = items < ctas ? items : ctas;
    if (grid_out) *grid_out = grid;
    k<<<grid, PL::NTH, PL::BYTES, s>>>(a, t);
    return cudaGetLastError();
}

template <int N, bool PK>
cudaError_t run_stage3z_variant(const StageArgs &a, const Tables<float> &t, cudaStream_t s, int *grid)
{
    static_assert(N == 1 || N == 3, "z-march lane groups exist for degrees 1 and 3");
    constexpr int T = N == 1 ? 8 : 4;  // 64 cells per plane at degree 1, 16 at degree 3
    if (a.av_on) {
        if (a.ns_on) return run_stage3z<N, true, true, T, T, PK>(a, t, s, grid);
        return run_stage3z<N, true, false, T, T, PK>(a, t, s, grid);
    }
    if (a.ns_on) return run_stage3z<N, false, true, T, T, PK>(a, t, s, grid);
    return run_stage3z<N, false, false, T, T, PK>(a, t, s, grid);
}

// the packed total-degree variants are instantiated in a translation unit of their own
// (dgx_inst_3d_packed_f32.cu), compiled in parallel with this one
template <int N>
cudaError_t run_stage3z_any(const StageArgs &a, const Tables<float> &t, cudaStream_t s, int *grid)
{
    if (a.cmap) return launch_stage3z_packed(N, a, t, s, grid);
    return run_stage3z_variant<N, false>(a, t, s, grid);
}

}  // namespace dgx

namespace dgx {

// Step prologue of the 3-D FP32-bulk plans of degrees 1 and 3 (runs with the limiter, where it cannot
// be folded into the first stage): the oscillation sensor and wiggle source of u^n (Sec. 4.1) and the
// per-CTA maxima of c_s and |v| at the Gauss points for the CFL step.  A cell per lane group, as in
// the z-marching stage kernel: the cell's modal x-lines in registers, modal -> nodal along x in
// registers and along y and z by lane products; no shared memory beyond the basis table, so many
// CTAs are resident and each lane group's loads of its next cell are in flight together.  CTA b
// takes the cells [b c, (b + 1) c) with c = ceil(ncell / gridDim.x), and writes partial b.
template <int N>
__global__ void __launch_bounds__(256) prologue3z_kernel(const PrologueArgs A, const Tables<float> Tg)
{
    constexpr int Q = N + 1, NP = Q * Q * Q, G = Q * Q, NC = 5, NTH = 256, NG = NTH / G;
    constexpr int VEC = (Q * 4) % 16 == 0 ? 16 : 8;
    __shared__ float tB[Q * Q];
    __shared__ double red[2][NTH / 32];
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gl = lane % G, grp = tid / G;
    const int ly = gl % Q, lz = gl / Q;
    for (int i = tid; i < Q * Q; i += NTH) tB[i] = Tg.B[i / Q][i % Q];
    if (tid == 0) s_bad = 0;
    __syncthreads();
    float by[Q], bz[Q];
    xcoef<Q>(tB, ly, by);
    xcoef<Q>(tB, lz, bz);
    // packed total-degree storage: the lane's modal x-line holds the modes l_x <= n - l_y - l_z
    const bool packed = A.cmap != nullptr;
    const int MS = packed ? A.ms : NP;
    const int plen = packed ? max(0, N + 1 - ly - lz) : Q;
    const int poff = packed ? (plen > 0 ? A.cmap[Q * (ly + Q * lz)] : 0) : gl * Q;
    const size_t fstride = (size_t)A.ncell * MS;
    const float *u = static_cast<const float *>(A.u);
    const float gamma = (float)A.gamma;
    const long long cpb = (A.ncell + gridDim.x - 1) / gridDim.x;
    const long long c0 = (long long)blockIdx.x * cpb;
    const long long c1 = c0 + cpb < A.ncell ? c0 + cpb : A.ncell;
    double cmax = 0.0, vmax = 0.0;
    int bad = 0;
    for (long long cb = c0; cb < c1; cb += NG) {  // the same trip count in every lane of the CTA
        const long long g = cb + grp;
        const bool valid = g < c1;
        float w[NC][Q];
        if (valid) {
            const size_t g0 = (size_t)g * MS + (size_t)poff;
#pragma unroll
            for (int f = 0; f < NC; ++f) z3_ld<Q, VEC>(u + g0 + f * fstride, packed, plen, w[f]);
        } else {
#pragma unroll
            for (int f = 0; f < NC; ++f)
#pragma unroll
                for (int m = 0; m < Q; ++m) w[f][m] = 0.0f;
        }
        if (A.update_sensor) {
            // sum of squares of the density modes, all and those the degree-(n-1) basis lacks
            float all = 0.0f, hi = 0.0f;
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                const bool top = A.total_degree ? (m + ly + lz == N) : (m == N || ly == N || lz == N);
                all += w[0][m] * w[0][m];
                if (top) hi += w[0][m] * w[0][m];
            }
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                all += __shfl_xor_sync(0xffffffffu, all, off);
                hi += __shfl_xor_sync(0xffffffffu, hi, off);
            }
            if (valid && gl == 0) {
                const double Sk = all > 0.0f ? (double)(hi / all) : 0.0;
                const double dt_prev = A.dtp[0], step = A.dtp[1];
                // S floored four decades below the onset threshold (its logarithm in FP32, as the sensor)
                const float sf = (float)(1e-4 * A.s_on);
                double dlog = 0.0;
                if (step > 0.0 && dt_prev > 0.0)
                    dlog = (double)((logf(fmaxf((float)Sk, sf)) - logf(fmaxf((float)A.S_prev[g], sf))) /
                                    (float)dt_prev);
                A.wig[g] = (Sk > A.s_on) ? A.f_w * fmax(0.0, dlog) : 0.0;
                A.S_prev[g] = Sk;
            }
        }
        // modal -> nodal: x in registers, then y and z across the group's lanes
#pragma unroll
        for (int f = 0; f < NC; ++f) {
            float o[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float acc = 0.0f;
#pragma unroll
                for (int m = 0; m < Q; ++m) acc = fmaf(Tg.B[i][m], w[f][m], acc);
                o[i] = acc;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) w[f][i] = xmatvec<Q, Q>(xmatvec<Q, 1>(o[i], by), bz);
        }
        if (valid) {
#pragma unroll
            for (int x = 0; x < Q; ++x) {
                float uu[NC], rho, v[3], p, cs;
#pragma unroll
                for (int f = 0; f < NC; ++f) uu[f] = w[f][x];
                if (!primitives<3>(uu, gamma, rho, v, p, cs)) bad = 1;
                cmax = fmax(cmax, (double)cs);
                vmax = fmax(vmax, (double)sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, off));
        vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    }
    if (lane == 0) {
        red[0][warp] = cmax;
        red[1][warp] = vmax;
    }
    if (bad) s_bad = 1;
    __syncthreads();
    if (tid == 0) {
        double c = 0.0, v = 0.0;
        for (int w = 0; w < NTH / 32; ++w) {
            c = fmax(c, red[0][w]);
            v = fmax(v, red[1][w]);
        }
        A.partial[2 * blockIdx.x + 0] = c;
        A.partial[2 * blockIdx.x + 1] = v;
        if (s_bad) atomicOr(A.status, DG_STATUS_NONPHYS);
    }
}

template <int N>
cudaError_t run_prologue3z(const PrologueArgs &a, const Tables<float> &t, cudaStream_t s)
{
    auto k = prologue3z_kernel<N>;
    static KernelSetup ks;
    cudaError_t e = kernel_setup(ks, k, 256, 0);
    if (e != cudaSuccess) return e;
    // one partial per tile of the general prologue's tiling (the count the time-step reduction reads)
    const int blocks = a.ntile[0] * a.ntile[1] * a.ntile[2];
    if (blocks == 0) return cudaSuccess;
    k<<<blocks, 256, 0, s>>>(a, t);
    return cudaGetLastError();
}

// prologue dispatch of the 3-D FP32-bulk unit: the lane-group prologue for degrees 1 and 3, the
// general tile prologue otherwise
template <int DIM, int N, typename Real, int TX, int TY, int TZ>
cudaError_t run_prologue_3d_f32_any(const PrologueArgs &a, const Tables<Real> &t, cudaStream_t s)
{
    if constexpr (DIM == 3 && std::is_same<Real, float>::value && (N == 1 || N == 3))
        return run_prologue3z<N>(a, t, s);
    else
        return run_prologue<DIM, N, Real, TX, TY, TZ>(a, t, s);
}

// stage dispatch of the 3-D FP32-bulk unit: the z-marching kernel for degrees 1 and 3 without a tracer,
// the general tile kernel otherwise
template <int DIM, int N, typename Real, int TX, int TY, int TZ, bool TRACER>
cudaError_t run_stage_3d_f32_any(const StageArgs &a, const Tables<Real> &t, cudaStream_t s, int *grid)
{
    if constexpr (DIM == 3 && std::is_same<Real, float>::value && (N == 1 || N == 3) && !TRACER)
        return run_stage3z_any<N>(a, t, s, grid);
    else
        return run_stage2_any<DIM, N, Real, TX, TY, TZ, TRACER>(a, t, s, grid);
}

}  // namespace dgx
