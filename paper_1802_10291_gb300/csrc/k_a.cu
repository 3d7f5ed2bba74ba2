// Kernel instantiations for FFT lengths: 2 4 8 16 32 64 6 12 24 48.
#include "mci_kernels.cuh"

namespace mci {

const void* kernel_lookup_a(int prec, bool cols, int N)
{
    switch (N) {
    MCI_KERNEL_CASE(2)
    MCI_KERNEL_CASE(4)
    MCI_KERNEL_CASE(8)
    MCI_KERNEL_CASE(16)
    MCI_KERNEL_CASE(32)
    MCI_KERNEL_CASE(64)
    MCI_KERNEL_CASE(6)
    MCI_KERNEL_CASE(12)
    MCI_KERNEL_CASE(24)
    MCI_KERNEL_CASE(48)
    }
    return nullptr;
}

__device__ bool device_launch_a(int prec, bool cols, int N, int grid, int smem, const KArgs& a)
{
    switch (N) {
    MCI_DEVICE_LAUNCH_CASE(2)
    MCI_DEVICE_LAUNCH_CASE(4)
    MCI_DEVICE_LAUNCH_CASE(8)
    MCI_DEVICE_LAUNCH_CASE(16)
    MCI_DEVICE_LAUNCH_CASE(32)
    MCI_DEVICE_LAUNCH_CASE(64)
    MCI_DEVICE_LAUNCH_CASE(6)
    MCI_DEVICE_LAUNCH_CASE(12)
    MCI_DEVICE_LAUNCH_CASE(24)
    MCI_DEVICE_LAUNCH_CASE(48)
    }
    return false;
}

}  // namespace mci
