// D3Q59 (Table I) instantiations of the step kernels: the h16 storage group.
// The lattice is split over several translation units so that they compile in parallel.
#include "lbm_kernels.cuh"

namespace lbm {

bool get_kernels_d3q59_h16(int storage, bool usolve_f64, bool read_pops, KernelTable* out)
{
    constexpr int L = 1;
    switch (storage) {
    case ST_F16_DEV:
        *out = usolve_f64 ? make_table<L, float, ST_F16_DEV, double>(read_pops)
                          : make_table<L, float, ST_F16_DEV, float>(read_pops);
        return true;
    case ST_BF16_DEV:
        *out = usolve_f64 ? make_table<L, float, ST_BF16_DEV, double>(read_pops)
                          : make_table<L, float, ST_BF16_DEV, float>(read_pops);
        return true;
    }
    return false;
}

}  // namespace lbm
