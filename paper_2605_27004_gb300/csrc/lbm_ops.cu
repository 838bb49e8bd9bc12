// Kernel instantiations of one (lattice, storage) pair. The build compiles this file once per
// pair with -DLBM_Q=<9|19|27> -DLBM_S=<0..3>, so the twelve objects build in parallel.
#include "lbm_launch.cuh"

#if !defined(LBM_Q) || !defined(LBM_S)
#error "compile with -DLBM_Q=<9|19|27> -DLBM_S=<0|1|2|3>"
#endif

#define LBM_CAT2(a, b, c, d) a##b##c##d
#define LBM_CAT(a, b, c, d) LBM_CAT2(a, b, c, d)

namespace lbm {
const Ops& LBM_CAT(ops_q, LBM_Q, _s, LBM_S)() { return Launch<LBM_Q, LBM_S>::ops(); }
}  // namespace lbm
