// Anisotropic advection-diffusion of a scalar phi (Sec. 1 and Sec. 5 name the transfer of the
// anisotropic equilibrium to advection-diffusion; the paper gives no equations for it).
//
// The populations g_i carry phi = sum_i g_i and relax by BGK towards the equilibrium of
// Eq. (3rd_order_equilibrium) taken with rho -> phi and the PRESCRIBED velocity u(x) of the
// carrier flow, so sum geq = phi, sum geq c = phi u and sum geq c c = phi (Theta + u u); with
// the Chapman-Enskog expansion of Sec. 3 this is d_t phi + div(phi u) = div((tau - 1/2) Theta
// grad phi) for a uniform u, i.e. the diffusion tensor is (tau - 1/2) Theta. Only phi is
// conserved, so the collision needs no moment other than the zeroth; the FP32 momentum identity
// of the flow kernels does not apply. Streaming, walls (half-way bounce-back: zero flux), the
// storage forms and the AA pattern are those of the flow kernels.
//
// The velocity is a [d][N] field in the arithmetic type (float, or double for FP64 storage),
// read once per cell, or absent (u = 0, pure anisotropic diffusion). These one-cell kernels
// serve FP32 / FP64 storage and boxes with walls; FP16 storage without walls runs the scalar
// collision in the two-cells-per-thread kernels of lbm_pairs.cuh (collide2 with ADE = true).
#pragma once
#include "lbm_kernels.cuh"

namespace lbm {
inline namespace LBM_VARIANT {

template <typename T>
struct VelField {
    const T* p[3];  // per-component planes of the advecting velocity; p[0] == nullptr: u = 0
};

// Relaxes d in place towards geq(phi, u(x)); returns phi - rho0 (phi0 of the shifted storage).
template <int Q, typename T>
__device__ __forceinline__ T ade_bgk(const Coef<T>& cf, const VelField<T>& vf, uint32_t n, T (&d)[Q]) {
    T ux = T(0), uy = T(0), uz = T(0);
    if (vf.p[0] != nullptr) {
        ux = ld_ro(vf.p[0] + n);
        uy = ld_ro(vf.p[1] + n);
        if (Lat<Q>::D == 3) uz = ld_ro(vf.p[2] + n);
    }
    T s = d[0];
#pragma unroll
    for (int k = 0; k < Lat<Q>::P; ++k) s += d[2 * k + 1] + d[2 * k + 2];
    const EqCell<T> e = eq_cell<T>(cf, s, cf.rho0 + s, ux, uy, uz);
    relax<Q, T>(cf, e, d);
    return s;
}

// Fused stream + collide of the scalar populations, two arrays, pull form (see k_step_pull).
template <int Q, int S, bool MASK>
__global__ void __launch_bounds__(256)
    k_ade_pull(Geom g, Coef<typename Store<S>::T> cf, VelField<typename Store<S>::T> vf,
               const Planes<const typename Store<S>::type> src, const Planes<typename Store<S>::type> dst,
               int* __restrict__ flag) {
    using T = typename Store<S>::T;
    Cell c;
    if (!make_cell(g, c)) return;
    const uint32_t lw = link_of<MASK>(g, c);
    // with walls, solid lanes of a sector that holds a fluid cell store zeros into their own
    // (never read) slots, so that destination sectors are written whole (as in k_step_pull)
    const bool solid = MASK && (lw & LINK_SOLID);
    const unsigned act = __activemask();
    if (MASK && __all_sync(act, solid)) return;
    T d[Q];
    if (MASK && __all_sync(act, lw == 0u)) {  // no wall link in the warp (see k_step_pull)
        gather<Q, S, false, LAYOUT_PULL, true>(c, 0u, cf, src, d);
    } else if (!solid) {
        gather<Q, S, MASK, LAYOUT_PULL, true>(c, lw, cf, src, d);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = T(0);
    }
    const T s = ade_bgk<Q, T>(cf, vf, c.n, d);
    if (!solid && !isfinite(s)) *flag = 1;
    if (MASK && !store_group<typename Store<S>::type>(act, solid)) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) st_raw(dst.p[i] + c.n, solid ? T(0) : from_shifted<S>(d[i], cf.so[i]));
}

// The scalar pull step with walls over the list of 32-byte sectors that hold a fluid cell (as
// k_step_pull_sectors for the flow; FP16 and FP32 storage).
template <int Q, int S>
__global__ void __launch_bounds__(256)
    k_ade_pull_sectors(Geom g, Coef<typename Store<S>::T> cf, CellList L, VelField<typename Store<S>::T> vf,
                       const Planes<const typename Store<S>::type> src, const Planes<typename Store<S>::type> dst,
                       int* __restrict__ flag) {
    using T = typename Store<S>::T;
    constexpr uint32_t G = 32u / sizeof(typename Store<S>::type);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t sec = t / G;
    uint32_t n = sec < L.count ? __ldg(L.idx + sec) * G + (t % G) : 0u;
    const bool valid = sec < L.count && n >= L.n_begin && n < L.n_end;
    if (!valid) n = L.n_begin;
    Cell c;
    make_cell_index(g, L, n, c);
    const uint32_t lw = valid ? __ldg(g.link + c.n) : LINK_SOLID;
    const bool solid = (lw & LINK_SOLID) != 0u;
    const unsigned act = __activemask();
    if (__all_sync(act, solid)) return;
    T d[Q];
    if (__all_sync(act, lw == 0u)) {
        gather<Q, S, false, LAYOUT_PULL, true>(c, 0u, cf, src, d);
    } else if (!solid) {
        gather<Q, S, true, LAYOUT_PULL, true>(c, lw, cf, src, d);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = T(0);
    }
    const T s = ade_bgk<Q, T>(cf, vf, c.n, d);
    if (!solid && !isfinite(s)) *flag = 1;
    const bool store = store_group<typename Store<S>::type>(act, solid);
    if (!valid || !store) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) st_raw(dst.p[i] + c.n, solid ? T(0) : from_shifted<S>(d[i], cf.so[i]));
}

// AA pattern in place (see k_step_aa): even steps read and write the own cell, odd steps the
// neighbours along +c_i.
template <int Q, int S, bool MASK, int ODD>
__global__ void __launch_bounds__(256)
    k_ade_aa(Geom g, Coef<typename Store<S>::T> cf, VelField<typename Store<S>::T> vf,
             const Planes<const typename Store<S>::type> src, const Planes<typename Store<S>::type> dst,
             int* __restrict__ flag) {
    using T = typename Store<S>::T;
    Cell c;
    if (!make_cell(g, c)) return;
    const uint32_t lw = link_of<MASK>(g, c);
    if (MASK && (lw & LINK_SOLID)) return;
    T d[Q];
    const bool clean = MASK && __all_sync(__activemask(), lw == 0u);  // see k_step_aa
    if (clean) {
        if (ODD)
            gather<Q, S, false, LAYOUT_AAODD, false>(c, 0u, cf, src, d);
        else
            gather<Q, S, false, LAYOUT_LOCAL, false>(c, 0u, cf, src, d);
    } else if (ODD) {
        gather<Q, S, MASK, LAYOUT_AAODD, false>(c, lw, cf, src, d);
    } else {
        gather<Q, S, MASK, LAYOUT_LOCAL, false>(c, lw, cf, src, d);
    }
    const T s = ade_bgk<Q, T>(cf, vf, c.n, d);
    if (!isfinite(s)) *flag = 1;
    if (clean)
        aa_store<Q, S, false, ODD>(c, 0u, cf, dst, d);
    else
        aa_store<Q, S, MASK, ODD>(c, lw, cf, dst, d);
}

}  // namespace LBM_VARIANT
}  // namespace lbm
