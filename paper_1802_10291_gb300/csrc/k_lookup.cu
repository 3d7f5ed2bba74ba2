// Joins the per-translation-unit kernel tables.
#include "mci_internal.h"

namespace mci {

const void* kernel_lookup_a(int prec, bool cols, int N);
const void* kernel_lookup_b(int prec, bool cols, int N);
const void* kernel_lookup_c(int prec, bool cols, int N);
const void* kernel_lookup_d(int prec, bool cols, int N);
const void* kernel_lookup_e(int prec, bool cols, int N);

const void* kernel_lookup(int prec, bool cols, int N)
{
    const void* (*tables[])(int, bool, int) = {kernel_lookup_a, kernel_lookup_b, kernel_lookup_c,
                                               kernel_lookup_d, kernel_lookup_e};
    for (auto t : tables)
        if (const void* k = t(prec, cols, N)) return k;
    return nullptr;
}

}  // namespace mci
