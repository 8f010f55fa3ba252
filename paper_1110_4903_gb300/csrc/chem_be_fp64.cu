// FP64 instantiations of the backward-Euler kernel (lanes per cell 2..32).
#include "chem_kernel.cuh"

namespace chem {

const void *be_kernel_fp64(int G) {
    switch (G) {
        case 2: return (const void *)&be_kernel<2, double>;
        case 4: return (const void *)&be_kernel<4, double>;
        case 8: return (const void *)&be_kernel<8, double>;
        case 16: return (const void *)&be_kernel<16, double>;
        case 32: return (const void *)&be_kernel<32, double>;
        default: return nullptr;
    }
}

}  // namespace chem
