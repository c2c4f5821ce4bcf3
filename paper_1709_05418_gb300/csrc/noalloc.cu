// noalloc.cu -- FP32 network forward that allocates no device memory.
//
// Its activation scratch is one file-scope __device__ array, so the call needs no
// context and never reaches cudaMalloc.  The array exists once per GPU that loads the
// library and lives until the process exits.  Host code must not hand the array's
// symbol to a kernel: in host code that name is only a stand-in, so the device address
// is looked up with cudaGetSymbolAddress, once per device, with that device current.
#include <mutex>

#include "common.cuh"

namespace rpnn {
namespace {

constexpr int64_t kStaticRows = RPNN_STATIC_MAX_ROWS;
constexpr int64_t kStaticFloats = 3 * kStaticRows * RPNN_H;   // o, F1 / tail, tail
__device__ __align__(256) float g_static_scratch[kStaticFloats];

constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

rpnn_status scratch_for_current_device(float** out) {
    int dev = 0;
    RPNN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) { set_error("device index %d out of range", dev); return RPNN_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        RPNN_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return RPNN_OK;
}

}  // namespace
}  // namespace rpnn

using namespace rpnn;

extern "C" rpnn_status rpnn_mlp_forward_f32_static(const float* dev_params, const float* dev_desc, int64_t q,
                                                   float* dev_out, void* stream) {
    set_error("%s", "");
    if (q < 0 || q > kStaticRows) {
        set_error("rpnn_mlp_forward_f32_static takes at most %lld rows (got %lld): its scratch is a fixed "
                  "static array",
                  (long long)kStaticRows, (long long)q);
        return RPNN_ERR_ARG;
    }
    if (q == 0) return RPNN_OK;
    if (!dev_params || !dev_desc || !dev_out) { set_error("null pointer"); return RPNN_ERR_ARG; }
    float* scratch = nullptr;
    rpnn_status st = scratch_for_current_device(&scratch);
    if (st) return st;
    // the context path's forward with no context: default GEMM tile, no split-K, no tuning
    const int64_t plane = kStaticRows * RPNN_H;
    float* const scr[3] = {scratch, scratch + plane, scratch + 2 * plane};
    const NetDims nd{&param_layout(), RPNN_DIN, RPNN_DESC_STRIDE};
    return rpnn_forward_f32(nullptr, nd, dev_params, dev_desc, q, nullptr, dev_out, nullptr, scr,
                            (cudaStream_t)stream);
}
