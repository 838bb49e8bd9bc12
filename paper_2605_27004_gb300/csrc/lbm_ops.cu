// Kernel instantiations of one (lattice, storage) pair. The build compiles this file once per
// pair with -DLBM_Q=<9|19|27> -DLBM_S=<0..4>, and once more per D3Q19 / D3Q27 pair with
// -DLBM_SLAB=1 for z-slab contexts, so the twenty-five objects build in parallel.
#include "lbm_launch.cuh"

#if !defined(LBM_Q) || !defined(LBM_S)
#error "compile with -DLBM_Q=<9|19|27> -DLBM_S=<0|1|2|3|4> [-DLBM_SLAB=1]"
#endif

#define LBM_CAT2(a, b, c, d, e) a##b##c##d##e
#define LBM_CAT(a, b, c, d, e) LBM_CAT2(a, b, c, d, e)
#if LBM_SLAB
#define LBM_OPS_NAME LBM_CAT(ops_q, LBM_Q, _s, LBM_S, _slab)
#else
#define LBM_OPS_NAME LBM_CAT(ops_q, LBM_Q, _s, LBM_S, )
#endif

namespace lbm {
const Ops& LBM_OPS_NAME() { return Launch<LBM_Q, LBM_S>::ops(); }
}  // namespace lbm
