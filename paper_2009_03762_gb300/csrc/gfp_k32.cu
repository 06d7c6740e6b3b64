// FP32 instantiation of the hot-path passes (bulk of the mixed-precision iteration).
#include "gfp_kimpl.cuh"
namespace gfp {
template struct Passes<float>;
template bool cz_cols_ok<float>(int, int);
template bool cz_tma_ok<float>(int, int);
template int cy_cols_max<float>(int);
}
