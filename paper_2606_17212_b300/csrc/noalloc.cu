// dgs_image_mse_noalloc: the per-image MSE / PSNR of dgs_image_mse for callers
// that cannot allocate memory.
//
// Some callers cannot call cudaMalloc or create a library context: code running
// inside a memory pool or arena they do not own, real-time loops where an
// allocation (and the device synchronisation cudaFree implies) is not allowed,
// or hosts that forbid the library from touching the allocator at all.  This
// entry point needs no context and allocates nothing: its only scratch (the
// FP64 partial sums) is the fixed file-scope device array below, which every
// GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <mutex>
#include <stdint.h>

#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int NOALLOC_MAX_PARTS = DGS_NOALLOC_MAX_PARTS;  // doubles of scratch

// Shared scratch of every call on a device; the last call's partial sums stay
// in it.  Host code must not pass &g_partial to a kernel (it is a host-side
// stand-in); it uses the device address from cudaGetSymbolAddress instead.
static __device__ __align__(256) double g_partial[NOALLOC_MAX_PARTS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double *g_partial_addr[MAX_DEVICES] = {};

// Device address of g_partial on the current device, looked up once per device.
cudaError_t scratch_address(int device, double **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partial_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partial);
        if (e != cudaSuccess) return e;
        g_partial_addr[device] = static_cast<double *>(p);
    }
    *out = g_partial_addr[device];
    return cudaSuccess;
}

// Variant of the MSE partial-sum kernel: reads the reference index from device
// memory and checks it (an out-of-range index turns that image's MSE into NaN).
// Same per-pixel FP32 squared error and FP64 chunk sums of MSE_CHUNK_PIX
// pixels as dgs_image_mse.  Every (image, chunk) partial is written exactly
// once per call, so the shared scratch needs no clearing between calls.
__global__ void __launch_bounds__(256) k_image_mse_noalloc(const float *__restrict__ images,
                                                           const float *__restrict__ refs,
                                                           const int32_t *__restrict__ ref_index, int n_refs,
                                                           size_t npix, float gscale, double *partial,
                                                           int parts, float *__restrict__ dL)
{
    __shared__ double wsum[8];
    const int s = blockIdx.y;
    const int r = ref_index[s];
    const bool ok = r >= 0 && r < n_refs;
    const float *im = images + (size_t)s * npix * 3;
    const float *rf = refs + (size_t)(ok ? r : 0) * npix * 3;
    double se = 0.0;
    const size_t base = (size_t)blockIdx.x * MSE_CHUNK_PIX;
    for (int k = 0; k < MSE_CHUNK_PIX / 256; ++k) {
        const size_t p = base + (size_t)k * 256 + threadIdx.x;
        if (p < npix) {
            float x[3], y[3];
            for (int c = 0; c < 3; ++c) { x[c] = im[3 * p + c]; y[c] = ok ? rf[3 * p + c] : 0.0f; }
            se += (double)pixel_sq_err(x[0], x[1], x[2], y[0], y[1], y[2]);
            if (dL)
                for (int c = 0; c < 3; ++c)
                    dL[((size_t)s * npix + p) * 3 + c] = ok ? gscale * (x[c] - y[c]) : __int_as_float(0x7fc00000);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = se;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += wsum[w];
        partial[(size_t)s * parts + blockIdx.x] = ok ? tot : __longlong_as_double(0x7ff8000000000000LL);
    }
}

__global__ void k_mse_reduce_noalloc(const double *partial, int S, int parts, double inv_count,
                                     double *__restrict__ mse, double *__restrict__ psnr)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= S) return;
    double acc = 0.0;
    for (int t = lane; t < parts; t += 32) acc += partial[(size_t)warp * parts + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const double m = acc * inv_count;
        mse[warp] = m;
        if (psnr) psnr[warp] = m > 0.0 ? 10.0 * log10(1.0 / m) : (m == 0.0 ? __longlong_as_double(0x7ff0000000000000LL) : m);
    }
}

}  // namespace
}  // namespace dgs

extern "C" int dgs_image_mse_noalloc(const float *images, const float *refs, const int32_t *ref_index, int S,
                                     int n_refs, int H, int W, float weight, double *mse, double *psnr,
                                     float *dL_dimages, dgs_stream stream)
{
    using namespace dgs;
    if (S < 0 || S > 65535 || H < 1 || W < 1 || n_refs < 1) return DGS_E_INVALID_ARG;
    if (S == 0) return DGS_OK;
    if (!images || !refs || !ref_index || !mse) return DGS_E_INVALID_ARG;
    const size_t npix = (size_t)H * (size_t)W, per = npix * 3;
    const size_t parts = (npix + MSE_CHUNK_PIX - 1) / MSE_CHUNK_PIX;
    if (parts > (size_t)NOALLOC_MAX_PARTS || (size_t)S * parts > (size_t)NOALLOC_MAX_PARTS)
        return DGS_E_SCRATCH;   // S * ceil(HW / 1024) must not exceed DGS_NOALLOC_MAX_PARTS
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= MAX_DEVICES) return DGS_E_CUDA;
    double *partial = nullptr;
    if (scratch_address(device, &partial) != cudaSuccess) return DGS_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const float gscale = (float)(2.0 * (double)weight / (double)per);
    dim3 grid((unsigned)parts, (unsigned)S);
    k_image_mse_noalloc<<<grid, 256, 0, st>>>(images, refs, ref_index, n_refs, npix, gscale, partial, (int)parts,
                                              dL_dimages);
    count_launch();
    const int threads = 256, blocks = (S * 32 + threads - 1) / threads;
    k_mse_reduce_noalloc<<<blocks, threads, 0, st>>>(partial, S, (int)parts, 1.0 / (double)per, mse, psnr);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DGS_OK : DGS_E_CUDA;
}
