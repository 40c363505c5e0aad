// D2Q21 (Table II) instantiations of the step kernels: the local-reference storages.
#include "lbm_kernels.cuh"

namespace lbm {

bool get_kernels_d2q21_loc(int storage, bool usolve_f64, bool read_pops, KernelTable* out)
{
    constexpr int L = 0;
    if (usolve_f64) return false;  // the local-reference storages run the u-solve in FP32 only
    switch (storage) {
    case ST_F32_LOC: *out = make_table<L, float, ST_F32_LOC, float>(read_pops); return true;
    case ST_F16_LOC: *out = make_table<L, float, ST_F16_LOC, float>(read_pops); return true;
    case ST_BF16_LOC: *out = make_table<L, float, ST_BF16_LOC, float>(read_pops); return true;
    }
    return false;
}

}  // namespace lbm
