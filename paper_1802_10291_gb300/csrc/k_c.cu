// Kernel instantiations for FFT lengths: 512 1024 384 768.
#include "mci_kernels.cuh"

namespace mci {

const void* kernel_lookup_c(int prec, bool cols, int N)
{
    switch (N) {
    MCI_KERNEL_CASE(512)
    MCI_KERNEL_CASE(1024)
    MCI_KERNEL_CASE(384)
    MCI_KERNEL_CASE(768)
    }
    return nullptr;
}

__device__ bool device_launch_c(int prec, bool cols, int N, int grid, int smem, const KArgs& a)
{
    switch (N) {
    MCI_DEVICE_LAUNCH_CASE(512)
    MCI_DEVICE_LAUNCH_CASE(1024)
    MCI_DEVICE_LAUNCH_CASE(384)
    MCI_DEVICE_LAUNCH_CASE(768)
    }
    return false;
}

}  // namespace mci
