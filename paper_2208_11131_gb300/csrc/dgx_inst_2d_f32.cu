// 2-D, FP32-bulk kernels.  Tiles: stage (TX,TY,1), prologue (TX,TY,1) per degree.
#define DGX_DIM 2
#define DGX_REAL float
#define DGX_SUFFIX 2d_f32
#define DGX_TILES(X) \
    X(0, 16, 16, 1, 16, 16, 1) X(1, 16, 8, 1, 16, 16, 1) X(2, 8, 8, 1, 16, 8, 1) \
    X(3, 6, 8, 1, 16, 8, 1) X(4, 6, 6, 1, 8, 8, 1) X(5, 5, 5, 1, 8, 4, 1)
// with a passive tracer (a sixth field): the tiles nearest those above that keep two CTAs per SM
#define DGX_TILES_TR(X) \
    X(0, 16, 16, 1, 16, 16, 1) X(1, 16, 7, 1, 16, 16, 1) X(2, 8, 8, 1, 16, 8, 1) \
    X(3, 6, 7, 1, 16, 8, 1) X(4, 6, 6, 1, 8, 8, 1) X(5, 5, 4, 1, 8, 4, 1)
#define DGX_STAGE_RUN run_stage2_any
#include "dgx_inst.cuh"
