// 2-D, FP32-bulk kernels.  Tiles: stage (TX,TY,1), prologue (TX,TY,1) per degree.
#define DGX_DIM 2
#define DGX_REAL float
#define DGX_SUFFIX 2d_f32
// (the tile autotuner, paper_2208_11131_gb300/autotune.py, builds its variants with both tables
// defined in a pre-included header, and writes its winners here)
#ifndef DGX_TILES
#define DGX_TILES(X) \
    X(0, 15, 16, 1, 16, 16, 1) X(1, 16, 8, 1, 16, 16, 1) X(2, 8, 8, 1, 16, 8, 1) \
    X(3, 7, 8, 1, 16, 8, 1) X(4, 7, 5, 1, 8, 8, 1) X(5, 5, 5, 1, 8, 4, 1)
#endif
// with a passive tracer (a sixth field): tiles that keep two CTAs per SM
#ifndef DGX_TILES_TR
#define DGX_TILES_TR(X) \
    X(0, 16, 16, 1, 16, 16, 1) X(1, 16, 6, 1, 16, 16, 1) X(2, 8, 8, 1, 16, 8, 1) \
    X(3, 6, 6, 1, 16, 8, 1) X(4, 7, 5, 1, 8, 8, 1) X(5, 4, 4, 1, 8, 4, 1)
#endif
#define DGX_STAGE_RUN run_stage_2d_f32_any
#include "dgx_stage2t.cuh"
#include "dgx_inst.cuh"
