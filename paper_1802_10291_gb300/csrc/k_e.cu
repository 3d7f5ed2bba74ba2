// Kernel instantiations for FFT lengths: 4096 3072.
#include "mci_kernels.cuh"

namespace mci {

const void* kernel_lookup_e(int prec, bool cols, int N)
{
    switch (N) {
    MCI_KERNEL_CASE(4096)
    MCI_KERNEL_CASE(3072)
    }
    return nullptr;
}

__device__ bool device_launch_e(int prec, bool cols, int N, int grid, int smem, const KArgs& a)
{
    switch (N) {
    MCI_DEVICE_LAUNCH_CASE(4096)
    MCI_DEVICE_LAUNCH_CASE(3072)
    }
    return false;
}

}  // namespace mci
