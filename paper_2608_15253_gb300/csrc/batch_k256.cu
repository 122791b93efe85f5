// Persistent replica-batch stage kernel, 256 threads per CTA.
#include "batch_dev.cuh"

namespace mm {

template __global__ void batch_stage_kernel<256>(BatchArgs a);

cudaError_t batch_kernel_attributes_256() {
    return cudaFuncSetAttribute(batch_stage_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024);  // room for the static work slot
}

void batch_kernel_launch_256(const BatchArgs& a, int blocks, size_t smem, cudaStream_t s) {
    batch_stage_kernel<256><<<blocks, 256, smem, s>>>(a);
}

int batch_kernel_occupancy_256(size_t smem) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_stage_kernel<256>, 256, smem);
    return nb;
}

}  // namespace mm
