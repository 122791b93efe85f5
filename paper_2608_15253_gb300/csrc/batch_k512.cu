// Persistent replica-batch stage kernel, 512 threads per CTA.
#include "batch_dev.cuh"

namespace mm {

template __global__ void batch_stage_kernel<512>(BatchArgs a);

cudaError_t batch_kernel_attributes_512() {
    return cudaFuncSetAttribute(batch_stage_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024);  // room for the static work slot
}

void batch_kernel_launch_512(const BatchArgs& a, int blocks, size_t smem, cudaStream_t s) {
    batch_stage_kernel<512><<<blocks, 512, smem, s>>>(a);
}

int batch_kernel_occupancy_512(size_t smem) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_stage_kernel<512>, 512, smem);
    return nb;
}

}  // namespace mm
