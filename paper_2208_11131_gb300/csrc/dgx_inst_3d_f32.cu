// 3-D, FP32-bulk kernels.
#define DGX_DIM 3
#define DGX_REAL float
#define DGX_SUFFIX 3d_f32
#define DGX_TILES(X) \
    X(0, 8, 4, 4, 8, 8, 4) X(1, 4, 4, 2, 8, 4, 4) X(2, 4, 2, 2, 4, 4, 4) \
    X(3, 2, 2, 2, 4, 4, 2) X(4, 2, 2, 1, 4, 2, 2) X(5, 2, 1, 1, 2, 2, 2)
#define DGX_STAGE_RUN run_stage_3d_f32_any
#define DGX_PROLOGUE_RUN run_prologue_3d_f32_any
#include "dgx_stage3z.cuh"
#include "dgx_inst.cuh"
