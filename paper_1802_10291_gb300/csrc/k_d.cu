// Kernel instantiations for FFT lengths: 2048 1536.
#include "mci_kernels.cuh"

namespace mci {

const void* kernel_lookup_d(int prec, bool cols, int N)
{
    switch (N) {
    MCI_KERNEL_CASE(2048)
    MCI_KERNEL_CASE(1536)
    }
    return nullptr;
}

__device__ bool device_launch_d(int prec, bool cols, int N, int grid, int smem, const KArgs& a)
{
    switch (N) {
    MCI_DEVICE_LAUNCH_CASE(2048)
    MCI_DEVICE_LAUNCH_CASE(1536)
    }
    return false;
}

}  // namespace mci
