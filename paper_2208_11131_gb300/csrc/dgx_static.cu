// dg_max_dt_noalloc: the CFL time step computed without allocating device memory.
//
// The ordinary path (dg_create + dg_max_dt) owns per-handle device buffers, among them the
// per-block maxima that the time-step reduction needs.  Some callers cannot let a library call
// cudaMalloc: applications that hand every byte of device memory to their own pool at start-up
// and forbid allocations afterwards, and time-stepping loops that cannot afford the implicit
// device synchronisation of cudaMalloc/cudaFree.  For them this entry point takes the state and
// the output from the caller and keeps its only scratch -- the per-block maxima and a status
// word -- in the file-scope array below, which every GPU that loads the library holds until the
// process exits.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "../../include/dgx.h"
#include "dgx_internal.h"

namespace {

constexpr int kStaticSlots = 1 << 18;  // per-block (max c_s, max |v|) pairs: 4 MiB
constexpr size_t kHeader = 256;      // status word, padded to keep the slots 256-byte aligned
constexpr size_t kScratchBytes = kHeader + sizeof(double) * 2 * (size_t)kStaticSlots;

static __device__ __align__(256) unsigned char g_cfl_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of g_cfl_scratch for the current device (looked up once per device)
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cfl_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// reduce the per-block maxima to dt = cfl h_min / (2 P (max c_s + max |v|)) (Eq. timestep);
// NaN when any Gauss point had rho <= 0 or p <= 0
__global__ void reduce_dt_static(int nblk, double cfl, double hmin, int P, double *dt_out)
{
    const int *status = reinterpret_cast<const int *>(g_cfl_scratch);
    const double *part = reinterpret_cast<const double *>(g_cfl_scratch + kHeader);
    __shared__ double rc[256], rv[256];
    double c = 0.0, v = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        c = fmax(c, part[2 * i]);
        v = fmax(v, part[2 * i + 1]);
    }
    rc[threadIdx.x] = c;
    rv[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            rc[threadIdx.x] = fmax(rc[threadIdx.x], rc[threadIdx.x + s]);
            rv[threadIdx.x] = fmax(rv[threadIdx.x], rv[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double dt = cfl * hmin / (2.0 * P * (rc[0] + rv[0]));
        *dt_out = (*status != 0 || !(dt > 0.0) || !isfinite(dt)) ? nan("") : dt;
    }
}

}  // namespace

extern "C" int dg_max_dt_noalloc(const dg_grid *grid, int degree, double gamma, double cfl, const double *dev_state,
                                 double *dev_dt, void *stream)
{
    using namespace dgx;
    if (!grid || !dev_state || !dev_dt || grid->dim < 2 || grid->dim > 3 || degree < 0 || degree > kMaxDegree ||
        !(gamma > 1.0) || !(cfl > 0.0))
        return DG_EINVAL;
    long long ncell = 1;
    double hmin = 1e300;
    int N[3] = {1, 1, 1};
    for (int a = 0; a < grid->dim; ++a) {
        if (grid->n[a] < 1 || !(grid->hi[a] > grid->lo[a])) return DG_EINVAL;
        N[a] = grid->n[a];
        ncell *= N[a];
        const double h = (grid->hi[a] - grid->lo[a]) / N[a];
        if (h < hmin) hmin = h;
    }
    if (ncell > 0x7fffffffLL) return DG_EINVAL;
    int st[3], pt[3];
    if (grid->dim == 2)
        tiles_2d_f64(degree, 0, st, pt);
    else
        tiles_3d_f64(degree, 0, st, pt);
    PrologueArgs a{};
    long long nblk = 1;
    for (int i = 0; i < 3; ++i) {
        a.N[i] = N[i];
        a.ntile[i] = (N[i] + pt[i] - 1) / pt[i];
        nblk *= a.ntile[i];
    }
    if (nblk > kStaticSlots) return DG_EUNSUPPORTED;  // more tiles than the static scratch holds

    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return DG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // the status word must start at zero on every call; the per-block slots are all overwritten
    if (cudaMemsetAsync(scratch, 0, sizeof(int), s) != cudaSuccess) return DG_ECUDA;
    a.gamma = gamma;
    a.nf = grid->dim + 2;
    a.ncell = ncell;
    a.u = dev_state;
    a.update_sensor = 0;
    a.partial = reinterpret_cast<double *>(static_cast<unsigned char *>(scratch) + kHeader);
    a.status = static_cast<int *>(scratch);
    Tables<double> td;
    Tables<float> tf;
    make_tables(degree, &td, &tf);
    cudaError_t e = grid->dim == 2 ? launch_prologue_2d_f64(degree, a, td, s) : launch_prologue_3d_f64(degree, a, td, s);
    if (e != cudaSuccess) return DG_ECUDA;
    reduce_dt_static<<<1, 256, 0, s>>>((int)nblk, cfl, hmin, degree + 1, dev_dt);
    if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
    return DG_OK;
}
