// FP64 instantiation of the chain: orbitals, FFTs, GEMM-like projections and Lanczos
// scalars all in double.
#include "chain.cuh"

namespace ll {
ChainBase* make_chain_f64() { return new Chain<double>(); }
}  // namespace ll
