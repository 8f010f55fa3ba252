// Request-server instantiations of the backward-Euler kernel (cells claimed
// from the server's device work queue), both precisions.
#include "../../include/chem.h"
#include "chem_kernel.cuh"

namespace chem {

const void *be_kernel_queue(int prec, int G) {
    if (prec == CHEM_MIXED) {
        switch (G) {
            case 2: return (const void *)&be_kernel<2, float, true>;
            case 4: return (const void *)&be_kernel<4, float, true>;
            case 8: return (const void *)&be_kernel<8, float, true>;
            case 16: return (const void *)&be_kernel<16, float, true>;
            case 32: return (const void *)&be_kernel<32, float, true>;
            default: return nullptr;
        }
    }
    switch (G) {
        case 2: return (const void *)&be_kernel<2, double, true>;
        case 4: return (const void *)&be_kernel<4, double, true>;
        case 8: return (const void *)&be_kernel<8, double, true>;
        case 16: return (const void *)&be_kernel<16, double, true>;
        case 32: return (const void *)&be_kernel<32, double, true>;
        default: return nullptr;
    }
}

}  // namespace chem
