// Kernel instantiations for FFT lengths: 128 256 96 192.
#include "mci_kernels.cuh"

namespace mci {

const void* kernel_lookup_b(int prec, bool cols, int N)
{
    switch (N) {
    MCI_KERNEL_CASE(128)
    MCI_KERNEL_CASE(256)
    MCI_KERNEL_CASE(96)
    MCI_KERNEL_CASE(192)
    }
    return nullptr;
}

__device__ bool device_launch_b(int prec, bool cols, int N, int grid, int smem, const KArgs& a)
{
    switch (N) {
    MCI_DEVICE_LAUNCH_CASE(128)
    MCI_DEVICE_LAUNCH_CASE(256)
    MCI_DEVICE_LAUNCH_CASE(96)
    MCI_DEVICE_LAUNCH_CASE(192)
    }
    return false;
}

}  // namespace mci
