// FP32 instantiation of the chain: orbitals, grids and FFTs in float; projections
// accumulated per warp in float and across warps in double; Lanczos scalars (norms, dots,
// beta/gamma/z) and the spectrum in double.
#include "chain.cuh"

namespace ll {
ChainBase* make_chain_f32() { return new Chain<float>(); }
}  // namespace ll
