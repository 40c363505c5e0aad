// D3Q59 (Table I) instantiations of the step kernels: the local-reference storages.
// The lattice is split over several translation units so that they compile in parallel.
#include "lbm_kernels.cuh"

namespace lbm {

bool get_kernels_d3q59_loc(int storage, bool usolve_f64, bool read_pops, KernelTable* out)
{
    constexpr int L = 1;
    if (usolve_f64) return false;  // the local-reference storages run the u-solve in FP32 only
    switch (storage) {
    case ST_F32_LOC: *out = make_table<L, float, ST_F32_LOC, float>(read_pops); return true;
    case ST_F16_LOC: *out = make_table<L, float, ST_F16_LOC, float>(read_pops); return true;
    case ST_BF16_LOC: *out = make_table<L, float, ST_BF16_LOC, float>(read_pops); return true;
    }
    return false;
}

}  // namespace lbm
