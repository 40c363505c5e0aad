// D3Q59 (Table I) instantiations of the step kernels: the f64 storage group.
// The lattice is split over several translation units so that they compile in parallel.
#include "lbm_kernels.cuh"

namespace lbm {

bool get_kernels_d3q59_f64(int storage, bool usolve_f64, bool read_pops, KernelTable* out)
{
    constexpr int L = 1;
    switch (storage) {
    case ST_F64:
        *out = make_table<L, double, ST_F64, double>(read_pops);
        return true;
    }
    return false;
}

}  // namespace lbm
