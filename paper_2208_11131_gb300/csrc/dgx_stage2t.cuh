// Lane-group tile kernel: the fused right-hand-side / Runge-Kutta stage for 2-D FP32-bulk grids whose
// degree has Q = n+1 a power of two (degrees 1 and 3), no tracer.
//
// The arithmetic is the collocated rewriting of the modal sums of Eq. time_stepping_final
// (dgx_kernels.cuh, header comment), organised like the 3-D z-marching kernel (dgx_stage3z.cuh):
// a cell's Q x-lines belong to Q lanes of one warp (lane gl of the group holds the x-line y = gl in
// registers), so the y passes of the modal<->nodal transforms, the nodal y-gradients and the weak
// divergence of the y fluxes are Q x Q products across the group's lanes (xor shuffles), and shared
// memory holds each cell's nodal values once, for the face phases.  A CTA works on a TX x TY tile of
// cells and its face-neighbour ring (2 (TX + TY) cells, half the tile's own cells at 8 x 8), looping
// over tiles.  Per tile: (L) load + transform tile and ring (fused first stage: sensor and wiggle
// source of the own cells); (R) recovered interface state at the face points (Navier-Stokes);
// (F) face fluxes; (V) per own cell and x-line: gradients, Euler - NS - AV flux at the line's Q
// nodes, weak divergence, sources, lifts of the four faces, nodal->modal transform and the epilogue.
// Faces on a tile boundary are computed by both tiles with the same code from the same data
// (bitwise equal on both sides: conservation without atomics).
#pragma once

#include "dgx_stage3z.cuh"

namespace dgx {

template <int N, bool AV, bool NS, int TX, int TY>
struct T2Plan {
    static constexpr int Q = N + 1, NP = Q * Q, G = Q;
    static constexpr int NTH = 256, NW = NTH / 32, CPW = 32 / G;
    static constexpr int NC = 4, NF = NC + (AV ? 1 : 0);
    static constexpr int TC = TX * TY, NH = 2 * (TX + TY);
    static_assert((Q & (Q - 1)) == 0 && Q <= 32, "lane groups need Q a power of two");
    static_assert(TC == NW * CPW, "one lane group per own cell of a tile");
    static constexpr int SLOT = NF * NP;  // floats per cell slot: [field][y][x]
    static constexpr int NSLOT = TC + NH;
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1), NFXY = NFX + NFY;
    static constexpr int FH = NC * NFXY * Q;           // face fluxes [field][face][point]
    static constexpr int UT = NS ? NC * NFXY * Q : 0;  // recovered state at the face points
    static constexpr int TAB = 64;
    static constexpr int OFF_FH = NSLOT * SLOT;
    static constexpr int OFF_UT = OFF_FH + FH;
    static constexpr int OFF_WIG = OFF_UT + UT;  // [cell] wiggle source
    static constexpr int OFF_TAB = OFF_WIG + TC;
    static constexpr int NREAL = OFF_TAB + 6 * TAB;
    static constexpr size_t BYTES = sizeof(float) * (size_t)NREAL + sizeof(int) * (size_t)NSLOT;
    static_assert((OFF_FH * 4) % 16 == 0 && (SLOT * 4) % 16 == 0, "vector accesses need 16-byte aligned arrays");
};

// the Q values of field f of a 2-D cell slot along axis a through face point p
// (a = 0: the x-line y = p; a = 1: the y-line x = p)
template <int Q, int a>
__device__ __forceinline__ void t2_axis_line(const float *slot, int f, int p, float (&v)[Q])
{
    constexpr int VEC = (Q * 4) % 16 == 0 ? 16 : 8;
    const float *b = slot + f * Q * Q;
    if constexpr (a == 0) {
        ld_line<Q, VEC>(b + p * Q, v);
    } else {
#pragma unroll
        for (int m = 0; m < Q; ++m) v[m] = b[m * Q + p];
    }
}

template <int Q, int a>
__device__ __forceinline__ void t2_recover(const float *sl, const float *sr, int p, const Tables<float> &Tg,
                                           float (&ut)[4])
{
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        float lv[Q], rv[Q];
        t2_axis_line<Q, a>(sl, f, p, lv);
        t2_axis_line<Q, a>(sr, f, p, rv);
        float acc = 0.0f;
#pragma unroll
        for (int m = 0; m < Q; ++m) acc = fmaf(Tg.Cm[m], lv[m], fmaf(Tg.Cp[m], rv[m], acc));
        ut[f] = acc;
    }
}

// flux through one face point normal to axis a, before weighting (the 2-D counterpart of
// z3_face_flux): HLLC of the traces minus the Navier-Stokes flux of the recovered state (tangential
// derivative gt) and the artificial-viscosity flux; an absent side (outflow boundary) gives the
// physical flux of the interior trace
template <int Q, bool AV, bool NS, int a>
__device__ __forceinline__ void t2_face_flux(const float *sl, const float *sr, int p, const float (&ut)[4],
                                             const float (&gt)[4], const Tables<float> &Tg, const StageArgs &A,
                                             float (&Fh)[4], int &bad)
{
    constexpr int NC = 4, NF = NC + (AV ? 1 : 0);
    constexpr bool GRAD = AV || NS;
    if (!sl || !sr) {
        const float *si = sl ? sl : sr;
        float u[NF], v[3], rho, pr_, cs;
#pragma unroll
        for (int f = 0; f < NC; ++f) {
            float q[Q];
            t2_axis_line<Q, a>(si, f, p, q);
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m < Q; ++m) acc = fmaf(sl ? Tg.Lp[m] : Tg.Lm[m], q[m], acc);
            u[f] = acc;
        }
        if (!primitives<2>(u, A.kf[SK_GAMMA], rho, v, pr_, cs)) bad = 1;
        euler_flux<2, false>(u, v, pr_, a, Fh);
        return;
    }
    float uL[NC + 1], uR[NC + 1], dn[NC];
    const float sc = Tg.inv_f * A.kf[SK_INV_H + a];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        float lv[Q], rv[Q];
        t2_axis_line<Q, a>(sl, f, p, lv);
        t2_axis_line<Q, a>(sr, f, p, rv);
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
    if (!hllc<2, false>(uL, uR, A.kf[SK_GAMMA], a, Fh, cL, cR)) bad = 1;
    if constexpr (NS) {
        float grd[2][NC];
#pragma unroll
        for (int f = 0; f < NC; ++f) {
            grd[a][f] = dn[f];
            grd[1 - a][f] = gt[f];
        }
        if (!(ut[0] > 0.0f)) bad = 1;
        float Fn[NC];
        ns_flux<2, false>(ut, grd, A.kf[SK_GAMMA], A.kf[SK_NU], A.kf[SK_KAPPA], 0.0f, a, Fn);
#pragma unroll
        for (int f = 0; f < NC; ++f) Fh[f] -= Fn[f];
    }
    if constexpr (AV) {
        const float eps = 0.5f * A.kf[SK_EPS] * (clamp01(uL[NC]) * cL + clamp01(uR[NC]) * cR);
#pragma unroll
        for (int f = 0; f < NC; ++f) Fh[f] -= eps * dn[f];
    }
}

// one face point of axis a (p: its index along the face), weighted for the lift, into sFh; with NS
// the recovered state and its tangential derivative come from sUt
template <int Q, bool AV, bool NS, int NFXY, int a>
__device__ __forceinline__ void t2_face(const float *sl, const float *sr, int face, int p, const float *sUt,
                                        const float *tDn, const float *tG, const Tables<float> &Tg,
                                        const StageArgs &A, float *sFh, int &bad)
{
    constexpr int NC = 4;
    float ut[NC], gt[NC];
    if (NS && sl && sr) {
#pragma unroll
        for (int f = 0; f < NC; ++f) {
            const float *pp = sUt + (f * NFXY + face) * Q;
            ut[f] = pp[p];
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m < Q; ++m) acc = fmaf(tDn[p * Q + m], pp[m], acc);
            gt[f] = acc * A.kf[SK_TWO_H + (1 - a)];
        }
    }
    float Fh[NC];
    t2_face_flux<Q, AV, NS, a>(sl, sr, p, ut, gt, Tg, A, Fh, bad);
    const float w = A.kf[SK_CAX + a] * tG[p];
#pragma unroll
    for (int f = 0; f < NC; ++f) sFh[(f * NFXY + face) * Q + p] = w * Fh[f];
}

template <int N, bool AV, bool NS, int TX, int TY>
__global__ void __launch_bounds__(256, 2) stage2t_kernel(const StageArgs A, const Tables<float> Tg)
{
    using PL = T2Plan<N, AV, NS, TX, TY>;
    constexpr int Q = PL::Q, NP = PL::NP, G = PL::G, NC = PL::NC, NF = PL::NF, TC = PL::TC, NH = PL::NH;
    constexpr int NFX = PL::NFX, NFXY = PL::NFXY, NTH = PL::NTH;
    constexpr int VEC = (Q * 4) % 16 == 0 ? 16 : 8;
    constexpr bool GRAD = AV || NS;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    float *sFh = sm + PL::OFF_FH, *sUt = sm + PL::OFF_UT, *sWig = sm + PL::OFF_WIG;
    float *tB = sm + PL::OFF_TAB, *tDn = tB + PL::TAB, *tWd = tDn + PL::TAB, *tG = tWd + PL::TAB;
    float *tLm = tG + PL::TAB, *tLp = tLm + PL::TAB;
    int *sG = reinterpret_cast<int *>(sm + PL::NREAL);
    __shared__ double s_red[2][NTH / 32];
    __shared__ double s_dt;
    __shared__ int s_status;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ly = lane % G;                     // the lane's x-line y within its cell
    const int grp = warp * PL::CPW + lane / G;   // own-cell index of the lane group within the tile

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
    const int N0 = A.N[0], N1 = A.N[1];
    const size_t fstride = (size_t)A.ncell * NP;

    float cmax = 0.0f, vmax = 0.0f;
    int bad = 0;

    auto gcell = [&](int o0, int o1, int cx, int cy) -> int {
        int gx = o0 + cx, gy = o1 + cy;
        if (gx < 0 || gx >= N0) {
            if (A.bc[0] != 0) return -1;
            gx = (gx + N0) % N0;
        }
        if (gy < 0 || gy >= N1) {
            if (A.bc[1] != 0) return -1;
            gy = (gy + N1) % N1;
        }
        return gx + N0 * gy;
    };

    // (L) one cell by one lane group: modal x-line y = ly of every field, x in registers, y across
    // the group's lanes; with `sensor` the oscillation sensor and wiggle source (fused first stage)
    auto load_cell = [&](float *slot, int g, bool sensor, float *wig_slot) {
        const bool valid = g >= 0;
        float w[NF][Q];
        if (valid) {
            const size_t g0 = (size_t)g * NP + (size_t)ly * Q;
#pragma unroll
            for (int f = 0; f < NF; ++f) ld_line<Q, VEC>(ub + g0 + f * fstride, w[f]);
            if (di) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    float dd[Q];
                    ld_line<Q, VEC>(di + g0 + f * fstride, dd);
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
            float all = 0.0f, hi = 0.0f;
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                const bool top = A.total_degree ? (m + ly == N) : (m == N || ly == N);
                all += w[0][m] * w[0][m];
                if (top) hi += w[0][m] * w[0][m];
            }
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                all += __shfl_xor_sync(0xffffffffu, all, off);
                hi += __shfl_xor_sync(0xffffffffu, hi, off);
            }
            if (valid && ly == 0) {
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
        } else if (AV && valid && ly == 0 && wig_slot) {
            *wig_slot = (float)A.wig[g];
        }
        float by[Q];
        xcoef<Q>(tB, ly, by);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            float o[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float acc = 0.0f;
#pragma unroll
                for (int m = 0; m < Q; ++m) acc = fmaf(Tg.B[i][m], w[f][m], acc);
                o[i] = xmatvec<Q, 1>(acc, by);
            }
            st_line<Q, VEC>(slot + f * NP + ly * Q, o);
        }
    };

    const int ntx = A.ntile[0], nty = A.ntile[1];
    const int ntiles = ntx * nty;
    float *halo = sm + TC * PL::SLOT;
    int *gHalo = sG + TC;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int o0 = (tile % ntx) * TX, o1 = (tile / ntx) * TY;
        const int V0 = min(TX, N0 - o0), V1 = min(TY, N1 - o1);
        const int mcx = grp % TX, mcy = grp / TX;
        const bool mine = mcx < V0 && mcy < V1;
        // (L) slot maps, then tile and ring
        if (tid < TC) {
            const int cx = tid % TX, cy = tid / TX;
            sG[tid] = (cx < V0 && cy < V1) ? gcell(o0, o1, cx, cy) : -1;
        } else if (tid < TC + NH) {
            const int h = tid - TC;
            int cx, cy;
            bool in;
            if (h < TY) {
                cx = -1, cy = h, in = cy < V1;
            } else if (h < 2 * TY) {
                cx = V0, cy = h - TY, in = cy < V1;
            } else if (h < 2 * TY + TX) {
                cx = h - 2 * TY, cy = -1, in = cx < V0;
            } else {
                cx = h - 2 * TY - TX, cy = V1, in = cx < V0;
            }
            gHalo[h] = in ? gcell(o0, o1, cx, cy) : -1;
        }
        __syncthreads();
        for (int t = grp; t < TC + NH; t += TC) {
            if (t < TC) load_cell(sm + t * PL::SLOT, sG[t], A.fused != 0, sWig + t);
            else load_cell(halo + (t - TC) * PL::SLOT, gHalo[t - TC], false, nullptr);
        }
        __syncthreads();

        auto slot_at = [&](int cx, int cy) -> const float * {
            if (cx >= 0 && cx < V0 && cy >= 0 && cy < V1) return sm + (cx + TX * cy) * PL::SLOT;
            int s;
            if (cx == -1) s = cy;
            else if (cx == V0) s = TY + cy;
            else if (cy == -1) s = 2 * TY + cx;
            else s = 2 * TY + TX + cx;
            return gHalo[s] >= 0 ? halo + s * PL::SLOT : nullptr;
        };
        auto face_of = [&](int q, int &a, const float *&sl, const float *&sr, int &face, int &p) -> bool {
            face = q / Q;
            p = q % Q;
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

        // (R) recovered state at the face points
        if (NS) {
            for (int q = tid; q < NFXY * Q; q += NTH) {
                int a, face, p;
                const float *sl, *sr;
                if (!face_of(q, a, sl, sr, face, p) || !sl || !sr) continue;
                float ut[NC];
                if (a == 0) t2_recover<Q, 0>(sl, sr, p, Tg, ut);
                else t2_recover<Q, 1>(sl, sr, p, Tg, ut);
#pragma unroll
                for (int f = 0; f < NC; ++f) sUt[(f * NFXY + face) * Q + p] = ut[f];
            }
            __syncthreads();
        }
        // (F) face fluxes, weighted for the lift
        for (int q = tid; q < NFXY * Q; q += NTH) {
            int a, face, p;
            const float *sl, *sr;
            if (!face_of(q, a, sl, sr, face, p)) continue;
            if (a == 0) t2_face<Q, AV, NS, NFXY, 0>(sl, sr, face, p, sUt, tDn, tG, Tg, A, sFh, bad);
            else t2_face<Q, AV, NS, NFXY, 1>(sl, sr, face, p, sUt, tDn, tG, Tg, A, sFh, bad);
        }
        __syncthreads();

        // (V) own cells
        {
            const float *slot = sm + grp * PL::SLOT;
            const int g = sG[grp];
            float u[NF][Q];
#pragma unroll
            for (int f = 0; f < NF; ++f) ld_line<Q, VEC>(slot + f * NP + ly * Q, u[f]);
            float dy[Q], wy[Q];
            xcoef<Q>(tDn, ly, dy);
            xcoef<Q>(tWd, ly, wy);
            const float gy = tG[ly];
            const float wig = AV ? sWig[grp] : 0.0f;
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
                float gr[2][NC];
                if (GRAD) {
#pragma unroll
                    for (int f = 0; f < NC; ++f) {
                        float acc = 0.0f;
#pragma unroll
                        for (int m = 0; m < Q; ++m) acc = fmaf(Tg.Dn[x][m], u[f][m], acc);
                        gr[0][f] = acc * K[SK_TWO_H + 0];
                        gr[1][f] = xmatvec<Q, 1>(u[f][x], dy) * K[SK_TWO_H + 1];
                    }
                }
                float rho, v[3], p, cs;
                if (!primitives<2>(uu, K[SK_GAMMA], rho, v, p, cs) && mine) bad = 1;
                if (A.fused && mine) {
                    cmax = fmaxf(cmax, cs);
                    vmax = fmaxf(vmax, sqrtf(v[0] * v[0] + v[1] * v[1]));
                }
                const float eps = AV ? K[SK_EPS] * clamp01(uu[NC]) * cs : 0.0f;
                float Fns[2][NC];
                if (NS) ns_flux_all<2>(uu, gr, K[SK_GAMMA], K[SK_NU], K[SK_KAPPA], Fns);
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    float F[NC];
                    euler_flux<2, false>(uu, v, p, a, F);
                    if (NS) {
#pragma unroll
                        for (int f = 0; f < NC; ++f) F[f] -= Fns[a][f];
                    }
                    if (AV) {
#pragma unroll
                        for (int f = 0; f < NC; ++f) F[f] -= eps * gr[a][f];
                    }
                    if (a == 0) {
                        const float w = K[SK_CAX + 0] * gy;
#pragma unroll
                        for (int f = 0; f < NC; ++f)
#pragma unroll
                            for (int i = 0; i < Q; ++i) r[f][i] = fmaf(Tg.Wd[i][x] * w, F[f], r[f][i]);
                    } else {
                        const float w = K[SK_CAX + 1] * Tg.G[x];
#pragma unroll
                        for (int f = 0; f < NC; ++f) r[f][x] += xmatvec<Q, 1>(w * F[f], wy);
                    }
                }
                const float Gv = Tg.G[x] * gy;
                if (force && mine) {
                    // driving source of Sec. 7.1: rho s into the momentum, s.(rho v) into the energy
                    const float wgt = 0.25f * Gv;
                    float se = 0.0f;
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        const float sa = force[((size_t)a * A.ncell + g) * NP + ly * Q + x];
                        r[1 + a][x] = fmaf(wgt * uu[0], sa, r[1 + a][x]);
                        se = fmaf(sa, uu[1 + a], se);
                    }
                    r[3][x] = fmaf(wgt, se, r[3][x]);
                }
                if (AV) {
                    float div = 0.0f;
#pragma unroll
                    for (int a = 0; a < 2; ++a) div += (gr[a][1 + a] - v[a] * gr[a][0]) / rho;
                    const float adot = K[SK_FV] * fmaxf(0.0f, -div) + wig - uu[NC] * cs * K[SK_INV_TAU];
                    r[NC][x] = 0.25f * Gv * adot;
                }
            }
            // lifts of the four face fluxes
            if (mine) {
                const int fxl = mcx + (TX + 1) * mcy;  // x-faces left / right: point y
                const int fyb = NFX + mcx + TX * mcy;  // y-faces bottom / top: points x
                const float lmy = tLm[ly], lpy = tLp[ly];
#pragma unroll
                for (int f = 0; f < NC; ++f) {
                    const float fL = sFh[(f * NFXY + fxl) * Q + ly];
                    const float fR = sFh[(f * NFXY + fxl + 1) * Q + ly];
                    float yb[Q], yt[Q];
                    ld_line<Q, VEC>(sFh + (f * NFXY + fyb) * Q, yb);
                    ld_line<Q, VEC>(sFh + (f * NFXY + fyb + TX) * Q, yt);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        float acc = r[f][i];
                        acc = fmaf(Tg.Lm[i], fL, acc);
                        acc = fmaf(-Tg.Lp[i], fR, acc);
                        acc = fmaf(lmy, yb[i], acc);
                        r[f][i] = fmaf(-lpy, yt[i], acc);
                    }
                }
            }
            // nodal -> modal: y across the group's lanes, x in registers
            float cy_[Q];
            xcoef<Q, true>(tB, ly, cy_);
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int i = 0; i < Q; ++i) r[f][i] = xmatvec<Q, 1>(r[f][i], cy_);
            if (mine) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const size_t gi = (size_t)f * fstride + (size_t)g * NP + (size_t)ly * Q;
                    constexpr int VD = (Q * 8) % 16 == 0 ? 16 : 8;
                    double uo[Q];
                    if (A.mode == 2) ld_line<Q, VD>(A.uold + gi, uo);
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
                            if (l + ly > N) L[l] = 0.0f;
                    }
                    if (A.mode == 0) {
#pragma unroll
                        for (int l = 0; l < Q; ++l) A.rhs_out[gi + l] = (double)L[l];
                        continue;
                    }
                    float din[Q], xv[Q], dnew[Q], zn_[Q];
                    if (di) {
                        ld_line<Q, VEC>(di + gi, din);
#pragma unroll
                        for (int l = 0; l < Q; ++l) din[l] = dsc * din[l];
                    } else {
#pragma unroll
                        for (int l = 0; l < Q; ++l) din[l] = 0.0f;
                    }
                    if (readx) {
                        ld_line<Q, VEC>(xb + gi, xv);
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
                    if (A.write_z) st_line<Q, VEC>(xb + gi, zn_);
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
                            st_line<Q, VEC>(A.uhi_new + gi, uf);
                        }
                    }
                }
            }
        }
        __syncthreads();
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

template <int N, bool AV, bool NS, int TX, int TY>
cudaError_t run_stage2t(const StageArgs &a_in, const Tables<float> &t, cudaStream_t s, int *grid_out)
{
    using PL = T2Plan<N, AV, NS, TX, TY>;
    auto k = stage2t_kernel<N, AV, NS, TX, TY>;
    static_assert(PL::BYTES <= 227 * 1024, "2-D lane-group tile exceeds shared memory");
    static KernelSetup ks;
    int sms = 0, per_sm = 0;
    cudaError_t e = kernel_setup(ks, k, PL::NTH, PL::BYTES, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    if (a_in.ntile[0] * a_in.ntile[1] * a_in.ntile[2] == 0) return cudaSuccess;  // set-up call
    StageArgs a = a_in;
    a.ntile[0] = (a.N[0] + TX - 1) / TX;
    a.ntile[1] = (a.N[1] + TY - 1) / TY;
    a.ntile[2] = 1;
    const int tiles = a.ntile[0] * a.ntile[1];
    const int ctas = sms * per_sm;
    const int grid = tiles < ctas ? tiles : ctas;
    if (grid_out) *grid_out = grid;
    k<<<grid, PL::NTH, PL::BYTES, s>>>(a, t);
    return cudaGetLastError();
}

template <int N>
cudaError_t run_stage2t_any(const StageArgs &a, const Tables<float> &t, cudaStream_t s, int *grid)
{
    static_assert(N == 1 || N == 3, "2-D lane groups exist for degrees 1 and 3");
    constexpr int TX = N == 1 ? 16 : 8, TY = 8;  // one lane group per own cell: 128 or 64 cells per tile
    if (a.av_on) {
        if (a.ns_on) return run_stage2t<N, true, true, TX, TY>(a, t, s, grid);
        return run_stage2t<N, true, false, TX, TY>(a, t, s, grid);
    }
    if (a.ns_on) return run_stage2t<N, false, true, TX, TY>(a, t, s, grid);
    return run_stage2t<N, false, false, TX, TY>(a, t, s, grid);
}

// stage dispatch of the 2-D FP32-bulk unit: the lane-group tile kernel for degrees 1 and 3 without a
// tracer, the general tile kernel otherwise
template <int DIM, int N, typename Real, int TX, int TY, int TZ, bool TRACER>
cudaError_t run_stage_2d_f32_any(const StageArgs &a, const Tables<Real> &t, cudaStream_t s, int *grid)
{
    if constexpr (DIM == 2 && std::is_same<Real, float>::value && (N == 1 || N == 3) && !TRACER)
        return run_stage2t_any<N>(a, t, s, grid);
    else
        return run_stage2_any<DIM, N, Real, TX, TY, TZ, TRACER>(a, t, s, grid);
}

}  // namespace dgx
