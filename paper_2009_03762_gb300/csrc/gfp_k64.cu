// FP64 instantiation of the hot-path passes.
#include "gfp_kimpl.cuh"
namespace gfp {
template struct Passes<double>;
template bool cz_cols_ok<double>(int, int);
template bool cz_tma_ok<double>(int, int);
template int cy_cols_max<double>(int);
}
