// D2Q21 (Table II) instantiations of the step kernels.
#include "lbm_kernels.cuh"

namespace lbm {

bool get_kernels_d2q21_loc(int storage, bool usolve_f64, bool read_pops, KernelTable* out);

bool get_kernels_d2q21(int storage, bool usolve_f64, bool read_pops, KernelTable* out)
{
    constexpr int L = 0;
    switch (storage) {
    case ST_F32:
        *out = usolve_f64 ? make_table<L, float, ST_F32, double>(read_pops) : make_table<L, float, ST_F32, float>(read_pops);
        return true;
    case ST_F32_DEV:
        *out = usolve_f64 ? make_table<L, float, ST_F32_DEV, double>(read_pops)
                          : make_table<L, float, ST_F32_DEV, float>(read_pops);
        return true;
    case ST_F16_DEV:
        *out = usolve_f64 ? make_table<L, float, ST_F16_DEV, double>(read_pops)
                          : make_table<L, float, ST_F16_DEV, float>(read_pops);
        return true;
    case ST_BF16_DEV:
        *out = usolve_f64 ? make_table<L, float, ST_BF16_DEV, double>(read_pops)
                          : make_table<L, float, ST_BF16_DEV, float>(read_pops);
        return true;
    case ST_F64:
        *out = make_table<L, double, ST_F64, double>(read_pops);
        return true;
    }
    return get_kernels_d2q21_loc(storage, usolve_f64, read_pops, out);
}

}  // namespace lbm
