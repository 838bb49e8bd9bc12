// Internal interface between the C-ABI host code (lbm_host.cu) and the kernel translation units
// (lbm_ops.cu, one object per lattice and storage). Not installed, not public.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Grid geometry as every kernel sees it. N < 2^31, so in-plane offsets are 32-bit.
// Every per-cell kernel processes the stored planes z0 .. nz - 1 - z0: all of them for a whole
// periodic box (z0 = 0); for a z-slab (z0 = 1) the interior planes between ghost plane 0 and ghost
// plane nz - 1, which hold the neighbouring slabs' boundary planes. Interior cells of a slab never
// wrap in z, so the wrapped offsets reach the ghost planes, which the halo exchange fills. z0 is
// not a field: each kernel object is compiled for one value (LBM_SLAB in the kernel headers; as a
// kernel parameter it changed the register allocation of the FP16 pair kernels).
struct Geom {
    int nx, ny, nz;
    uint32_t N;            // nx*ny*nz (stored cells, ghost planes included)
    const uint32_t* link;  // per-cell link words or null (all fluid): bit i set when the
                           // neighbour x - c_i is solid, bit 31 set when x itself is solid
};
constexpr uint32_t LINK_SOLID = 0x80000000u;

// The fluid cells of a box with walls, listed in increasing cell index, so that a kernel can give
// every lane of a warp a fluid cell (FP16 AA steps); or, for the FP16 pull step, the 16-cell
// groups (one 32-byte sector of every FP16 plane) that hold at least one fluid cell (rows of the porous medium are about 30 % solid, and a lane
// of a solid cell still issues every instruction of its warp). A cell's coordinates come back
// from its index by exact reciprocal multiplication: n / d = umul64hi(n, ceil(2^64 / d)) for
// n, d < 2^32 and d >= 2.
struct CellList {
    const uint32_t* idx;
    uint32_t count;
    unsigned long long rnx, rnxy;  // ceil(2^64 / nx), ceil(2^64 / (nx ny))
    uint32_t n_begin, n_end;       // the processed cells (interior planes): n_begin <= n < n_end
};

// Per-run constants, derived on the host in FP64 from (tau, Theta, rho0, order) and rounded
// once to the arithmetic type T. Arrays are indexed by the library's direction order.
template <typename T>
struct Coef {
    T omega;      // 1/tau
    T rho0;       // reference density of the shifted representation
    T c3;         // 9/2 for the third-order equilibrium, 0 for the second order
    T K[6];       // K~ = Theta - cs2 I: xx, yy, zz, xy, xz, yz
    T r[27];      // rest equilibrium r_i = w_i rho0 (1 + 9/2 h_i)
    T so[27];     // storage offset: stored value = f_i - r_i + so_i (so = r for plain storage,
                  // 0 for the r-shifted forms, r_i - w_i rho0 for the w-shifted FP16 form)
    T A[27];      // w_i (1 + 9/2 h_i): density coefficient of the even part
    T B[27];      // w_i (3 + 3 c3 h_i): linear coefficient of the odd part
    T h[27];      // h_i = c_i.K~.c_i - cs2 tr K~
    T Pirest[6];  // sum_i r_i c_ia c_ib = rho0 Theta_ab
};

// Where the pre-collision population f_i(x, t) of the current state lives:
//   LOCAL  f_i(x) = A[i][x]                                  (AA pattern, even step count)
//   PULL   f_i(x) = S[i][x - c_i], or S[opp i][x] if x - c_i is solid   (two-array pull)
//   AAODD  f_i(x) = A[opp i][x - c_i], or A[i][x] if x - c_i is solid (AA, odd step count)
enum Layout { LAYOUT_LOCAL = 0, LAYOUT_PULL = 1, LAYOUT_AAODD = 2 };

// Launch shape shared by every per-cell kernel: 256-thread blocks, x fastest, one grid plane per
// processed lattice plane (nzp of them).
struct Shape {
    dim3 grid, block;
    long long nblocks;
};
Shape shape_for(const Geom& g, int nzp);

// Block width for n threads along x: a multiple of 32 up to 256 that wastes the fewest threads
// in the last block of a row; among those, a divisor of 256 (so that blocks of bx x 256/bx
// threads stay full: a kernel limited to two blocks per SM by its registers keeps 16 warps),
// then the widest. 384 threads per row run as three 128 x 2 blocks instead of two 256-thread
// blocks a quarter of which idle; 192 as 64 x 4 rather than 192 x 1.
inline int block_x_for(int n, int threads = 256) {
    int best = 32, waste = 1 << 30;
    bool full = true;
    for (int bx = threads; bx >= 32; bx -= 32) {
        const int w = ((n + bx - 1) / bx) * bx - n;
        const bool f = threads % bx == 0;
        if (w < waste || (w == waste && f && !full)) {
            waste = w;
            best = bx;
            full = f;
        }
    }
    return best;
}

// Kernel launchers of one (lattice, storage) pair. `coef` points at a Coef<double> (storage
// LBM_FP64) or a Coef<float> (every other storage). Field pointers (rho, u, Pi, f, grad, lam,
// du0) are double for FP64 and float otherwise; population pointers have the storage type.
struct Ops {
    cudaError_t (*init)(const Geom&, const void* coef, int layout, const void* rho, const void* u, void* dst,
                        cudaStream_t);
    cudaError_t (*step_pull)(const Geom&, const void* coef, const void* src, void* dst, int* flag, cudaStream_t);
    cudaError_t (*step_aa)(const Geom&, const void* coef, int odd, const void* src, void* dst, int* flag,
                           cudaStream_t);
    // the pull step over a list of 32-byte sectors (boxes with walls, FP16 and FP32 storage) and
    // the AA step over a fluid-cell list (boxes with walls, FP16 storage)
    cudaError_t (*step_pull_sectors)(const Geom&, const void* coef, const CellList&, const void* src, void* dst,
                                     int* flag, cudaStream_t);
    cudaError_t (*step_aa_list)(const Geom&, const void* coef, const CellList&, int odd, const void* src, void* dst,
                                int* flag, cudaStream_t);
    cudaError_t (*moments)(const Geom&, const void* coef, int layout, const void* src, void* rho, void* u, void* Pi,
                           void* f, cudaStream_t);
    cudaError_t (*totals)(const Geom&, const void* coef, int layout, const void* src, double* partials, int* flag,
                          cudaStream_t);
    cudaError_t (*adj_seed)(const Geom&, const void* coef, int layout, const void* src, const void* grad, void* lam,
                            cudaStream_t);
    cudaError_t (*adj_step)(const Geom&, const void* coef, int layout, const void* src, const void* lam_next,
                            void* lam, double* gpart, cudaStream_t);
    cudaError_t (*adj_init)(const Geom&, const void* coef, const void* rho0, const void* u0, const void* lam0,
                            void* du0, double* gpart, cudaStream_t);
    // link words from a byte mask (device, N bytes, nonzero = solid)
    cudaError_t (*link_mask)(const Geom&, const uint8_t* solid, uint32_t* link, cudaStream_t);
    // one advection-diffusion step (lbm_ade.cuh); u is the [d][N] advecting velocity in the
    // field type, or null for u = 0
    cudaError_t (*ade_pull)(const Geom&, const void* coef, const void* u, const void* src, void* dst, int* flag,
                            cudaStream_t);
    cudaError_t (*ade_aa)(const Geom&, const void* coef, const void* u, int odd, const void* src, void* dst,
                          int* flag, cudaStream_t);
    // the scalar pull step over the sector list (boxes with walls, FP16 and FP32 storage)
    cudaError_t (*ade_pull_sectors)(const Geom&, const void* coef, const CellList&, const void* u, const void* src,
                                    void* dst, int* flag, cudaStream_t);
};

// One translation unit per (lattice, storage): lbm_ops.cu compiled with LBM_Q / LBM_S, and for
// D3Q19 / D3Q27 once more with LBM_SLAB = 1 for z-slab contexts (ops_q<Q>_s<S>_slab).
#define LBM_OPS_DECL(Q, S) const Ops& ops_q##Q##_s##S(); const Ops& ops_q##Q##_s##S##_slab();
const Ops& ops_q9_s0(); const Ops& ops_q9_s1(); const Ops& ops_q9_s2(); const Ops& ops_q9_s3(); const Ops& ops_q9_s4();
LBM_OPS_DECL(19, 0) LBM_OPS_DECL(19, 1) LBM_OPS_DECL(19, 2) LBM_OPS_DECL(19, 3) LBM_OPS_DECL(19, 4)
LBM_OPS_DECL(27, 0) LBM_OPS_DECL(27, 1) LBM_OPS_DECL(27, 2) LBM_OPS_DECL(27, 3) LBM_OPS_DECL(27, 4)
#undef LBM_OPS_DECL

// Deterministic FP64 sum of `nb` partial records of `width` doubles into out[width]
// (one block, fixed order).
cudaError_t reduce_partials(const double* partials, long long nb, int width, double* out, cudaStream_t s);

}  // namespace lbm
