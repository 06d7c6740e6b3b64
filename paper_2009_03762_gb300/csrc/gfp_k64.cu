// FP64 instantiation of the hot-path passes.
#include "gfp_kimpl.cuh"
namespace gfp {
template struct Passes<double>;
}
