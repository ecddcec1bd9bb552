// tiDAS as per-row Toeplitz GEMMs on tcgen05 tensor cores (placeholder until
// the tensor-core path lands).
#include "common.cuh"

namespace tidas {
// Written by bounded waits of the tensor-core kernels; read by tidas_device_status.
__device__ int g_wait_error = 0;

int launch_tidas_gemm(const float*, int, int, bool, int, int, const void*, float*, int, bool,
                      cudaStream_t) {
    return set_error(TIDAS_ERR_UNSUPPORTED, "tidas GEMM variants not built yet");
}
}  // namespace tidas

extern "C" int tidas_device_status(int32_t* status) {
    TIDAS_REQUIRE(status, "tidas_device_status: null argument");
    TIDAS_CUDA(cudaDeviceSynchronize());
    int v = 0, zero = 0;
    TIDAS_CUDA(cudaMemcpyFromSymbol(&v, tidas::g_wait_error, sizeof(int)));
    TIDAS_CUDA(cudaMemcpyToSymbol(tidas::g_wait_error, &zero, sizeof(int)));
    *status = v;
    if (v != 0)
        return tidas::set_error(TIDAS_ERR_TIMEOUT, "a bounded device wait gave up (code %d)", v);
    return TIDAS_OK;
}
