// Explicit instantiation of the stage and prologue kernels for one
// (dimension, precision) pair.  The including unit defines
//   DGX_DIM, DGX_REAL, DGX_SUFFIX and DGX_TILES(X) with one
//   X(degree, stage TX,TY,TZ, prologue TX,TY,TZ) entry per degree 0..5, and optionally
//   DGX_TILES_TR(X), the stage tiles of the plans with a passive tracer (same form; the prologue
//   entries are not used: the prologue tiles are those of DGX_TILES).
#include "dgx_limiter.cuh"
#include "dgx_stage2.cuh"

// DGX_STAGE_RUN names the stage dispatch of the unit (run_stage2_any: the persistent, line-oriented
// stage kernel)

#ifndef DGX_TILES_TR
#define DGX_TILES_TR(X) DGX_TILES(X)
#endif
// DGX_PROLOGUE_RUN names the step-prologue dispatch of the unit (run_prologue: the tile prologue)
#ifndef DGX_PROLOGUE_RUN
#define DGX_PROLOGUE_RUN run_prologue
#endif

#define DGX_CAT2(a, b) a##b
#define DGX_CAT(a, b) DGX_CAT2(a, b)

namespace dgx {

#define DGX_STAGE_CASE(n, sx, sy, sz, px, py, pz) \
    case n:                                       \
        return DGX_STAGE_RUN<DGX_DIM, n, DGX_REAL, sx, sy, sz, false>(a, t, s, grid);
#define DGX_STAGE_CASE_TR(n, sx, sy, sz, px, py, pz) \
    case n:                                          \
        return DGX_STAGE_RUN<DGX_DIM, n, DGX_REAL, sx, sy, sz, true>(a, t, s, grid);
#define DGX_PRO_CASE(n, sx, sy, sz, px, py, pz) \
    case n:                                     \
        return DGX_PROLOGUE_RUN<DGX_DIM, n, DGX_REAL, px, py, pz>(a, t, s);
#define DGX_BATCH_CASE(n, sx, sy, sz, px, py, pz) \
    case n:                                      \
        return run_stage2_batch_any<DGX_DIM, n, DGX_REAL, sx, sy, sz>(av, ns, descs, tile_off, nsims, total, t, s);
#define DGX_LIM_CASE(n, sx, sy, sz, px, py, pz) \
    case n:                                    \
        return run_limiter_any<DGX_DIM, n, DGX_REAL>(a, t, s);
#define DGX_TILE_CASE(n, sx, sy, sz, px, py, pz) \
    case n:                                      \
        st[0] = sx;                              \
        st[1] = sy;                              \
        st[2] = sz;                              \
        pr[0] = px;                              \
        pr[1] = py;                              \
        pr[2] = pz;                              \
        break;
#define DGX_STILE_CASE(n, sx, sy, sz, px, py, pz) \
    case n:                                       \
        st[0] = sx;                               \
        st[1] = sy;                               \
        st[2] = sz;                               \
        break;

cudaError_t DGX_CAT(launch_stage_, DGX_SUFFIX)(int degree, const StageArgs &a, const Tables<DGX_REAL> &t,
                                               cudaStream_t s, int *grid)
{
    if (a.tracer_on) {
        switch (degree) { DGX_TILES_TR(DGX_STAGE_CASE_TR) }
    } else {
        switch (degree) { DGX_TILES(DGX_STAGE_CASE) }
    }
    return cudaErrorInvalidValue;
}

cudaError_t DGX_CAT(launch_prologue_, DGX_SUFFIX)(int degree, const PrologueArgs &a, const Tables<DGX_REAL> &t,
                                                  cudaStream_t s)
{
    switch (degree) { DGX_TILES(DGX_PRO_CASE) }
    return cudaErrorInvalidValue;
}

cudaError_t DGX_CAT(launch_stage_batch_, DGX_SUFFIX)(int degree, int av, int ns, const StageArgs *descs,
                                                     const int *tile_off, int nsims, int total,
                                                     const Tables<DGX_REAL> &t, cudaStream_t s)
{
    switch (degree) { DGX_TILES(DGX_BATCH_CASE) }
    return cudaErrorInvalidValue;
}

cudaError_t DGX_CAT(launch_limiter_, DGX_SUFFIX)(int degree, const LimiterArgs &a, const Tables<DGX_REAL> &t,
                                                 cudaStream_t s)
{
    switch (degree) { DGX_TILES(DGX_LIM_CASE) }
    return cudaErrorInvalidValue;
}

void DGX_CAT(tiles_, DGX_SUFFIX)(int degree, int tracer, int *st, int *pr)
{
    st[0] = st[1] = st[2] = pr[0] = pr[1] = pr[2] = 0;
    switch (degree) { DGX_TILES(DGX_TILE_CASE) }
    if (tracer) {
        switch (degree) { DGX_TILES_TR(DGX_STILE_CASE) }
    }
}

}  // namespace dgx
