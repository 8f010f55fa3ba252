// Mixed-precision instantiations: Jacobian, LU and solve in FP32; rates,
// sources, residual, update and temperature in FP64.
#include "chem_kernel.cuh"

namespace chem {

const void *be_kernel_mixed(int G) {
    switch (G) {
        case 2: return (const void *)&be_kernel<2, float>;
        case 4: return (const void *)&be_kernel<4, float>;
        case 8: return (const void *)&be_kernel<8, float>;
        case 16: return (const void *)&be_kernel<16, float>;
        case 32: return (const void *)&be_kernel<32, float>;
        default: return nullptr;
    }
}

}  // namespace chem
