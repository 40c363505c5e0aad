// D3Q59 (Table I) instantiations of the step kernels: the f32 storage group.
// The lattice is split over several translation units so that they compile in parallel.
#include "lbm_kernels.cuh"

namespace lbm {

bool get_kernels_d3q59_f32(int storage, bool usolve_f64, bool read_pops, KernelTable* out)
{
    constexpr int L = 1;
    switch (storage) {
    case ST_F32:
        *out = usolve_f64 ? make_table<L, float, ST_F32, double>(read_pops) : make_table<L, float, ST_F32, float>(read_pops);
        return true;
    case ST_F32_DEV:
        *out = usolve_f64 ? make_table<L, float, ST_F32_DEV, double>(read_pops)
                          : make_table<L, float, ST_F32_DEV, float>(read_pops);
        return true;
    }
    return false;
}

}  // namespace lbm

namespace lbm {

bool get_kernels_d3q59_h16(int storage, bool usolve_f64, bool read_pops, KernelTable* out);
bool get_kernels_d3q59_f64(int storage, bool usolve_f64, bool read_pops, KernelTable* out);
bool get_kernels_d3q59_loc(int storage, bool usolve_f64, bool read_pops, KernelTable* out);

bool get_kernels_d3q59(int storage, bool usolve_f64, bool read_pops, KernelTable* out)
{
    return get_kernels_d3q59_f32(storage, usolve_f64, read_pops, out) ||
           get_kernels_d3q59_h16(storage, usolve_f64, read_pops, out) ||
           get_kernels_d3q59_f64(storage, usolve_f64, read_pops, out) ||
           get_kernels_d3q59_loc(storage, usolve_f64, read_pops, out);
}

}  // namespace lbm
