// Host-side launchers of one (lattice, storage) pair: kernel choice (one or two cells per
// thread), launch shapes and the dispatch over walls and layouts.
#pragma once
#include "lbm_ade.cuh"
#include "lbm_kernels.cuh"
#include "lbm_adjoint2.cuh"
#include "lbm_pairs.cuh"
#include "lbm_quads.cuh"

namespace lbm {
inline namespace LBM_VARIANT {

// ---------------------------------------------------------------------------------------------
template <int Q, int S>
struct Launch {
    using ST = typename Store<S>::type;
    using T = typename Store<S>::T;
    using CF = Coef<T>;
    static Planes<const ST> cpl(const void* p, const Geom& g) { return planes_of(static_cast<const ST*>(p), Q, g.N); }
    static Planes<ST> mpl(void* p, const Geom& g) { return planes_of(static_cast<ST*>(p), Q, g.N); }
    static Planes<const T> cfl(const void* p, const Geom& g) { return planes_of(static_cast<const T*>(p), Q, g.N); }
    static Planes<T> mfl(void* p, const Geom& g) { return planes_of(static_cast<T*>(p), Q, g.N); }

    static cudaError_t init(const Geom& g, const void* coef, int layout, const void* rho, const void* u, void* dst,
                            cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        auto r = static_cast<const T*>(rho);
        auto uu = static_cast<const T*>(u);
        const auto o = mpl(dst, g);
        const bool m = g.link != nullptr;
        if (layout == LAYOUT_PULL) {
            if (m)
                k_init<Q, S, true, LAYOUT_PULL><<<sh.grid, sh.block, 0, st>>>(g, cf, r, uu, o);
            else
                k_init<Q, S, false, LAYOUT_PULL><<<sh.grid, sh.block, 0, st>>>(g, cf, r, uu, o);
        } else {
            if (m)
                k_init<Q, S, true, LAYOUT_LOCAL><<<sh.grid, sh.block, 0, st>>>(g, cf, r, uu, o);
            else
                k_init<Q, S, false, LAYOUT_LOCAL><<<sh.grid, sh.block, 0, st>>>(g, cf, r, uu, o);
        }
        return cudaGetLastError();
    }

    // Two cells per thread pay off where the one-cell kernel is instruction-bound: FP16 storage
    // without walls (measured at 256^3: D3Q19 0.61 -> 0.82, D3Q27 0.70 -> 0.83 of the copy peak,
    // the D3Q27 kernels in 128-thread blocks, see pair_threads).
    // FP32 storage is at the bandwidth bound with one cell per thread already, and the wall
    // variants lose occupancy.
    static bool pairs(const Geom& g) { return S == 3 && !g.link && (g.nx % 2) == 0; }
    // Four cells per thread (lbm_quads.cuh) for FP16 D2Q9 / D3Q19 without walls when every warp of
    // a row is full (nx a multiple of 128): measured at 256^3 / 512^3 pull 0.84 -> 0.93 / 0.86 ->
    // 0.96 of the copy peak, AA 0.79 -> 0.84 / 0.81 -> 0.86; at 64^3 (16 threads per row, half of
    // every warp idle) the two-cell kernels stay faster. D3Q27 would need 108 live FP32
    // populations per thread and stays at two cells.
    static bool quads(const Geom& g) { return S == 3 && Q != 27 && !g.link && (g.nx % 128) == 0; }

    static cudaError_t step_pull(const Geom& g, const void* coef, const void* src, void* dst, int* flag,
                                 cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        const auto a = cpl(src, g);
        const auto b = mpl(dst, g);
        if constexpr (S == 3) {  // pairs(g) holds for FP16 r-shifted storage only
            if constexpr (Q != 27) {
                if (quads(g)) {
                    const Shape sq = shape_quads(g);
                    k_step_pull4<Q><<<sq.grid, sq.block, 0, st>>>(g, cf, VelField<float>{}, a, b, flag);
                    return cudaGetLastError();
                }
            }
            if (pairs(g)) {
                const Shape sp = shape_pairs(g, pair_threads<Q>());
                k_step_pull2<Q, S, false><<<sp.grid, sp.block, 0, st>>>(g, cf, VelField<float>{}, a, b, flag);
                return cudaGetLastError();
            }
        }
        if (g.link)
            k_step_pull<Q, S, true><<<sh.grid, sh.block, 0, st>>>(g, cf, a, b, flag);
        else
            k_step_pull<Q, S, false><<<sh.grid, sh.block, 0, st>>>(g, cf, a, b, flag);
        return cudaGetLastError();
    }

    static cudaError_t step_aa(const Geom& g, const void* coef, int odd, const void* src, void* dst, int* flag,
                               cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        const auto a = cpl(src, g);
        const auto b = mpl(dst, g);
        if constexpr (S == 3) {  // pairs(g) holds for FP16 r-shifted storage only
            // no walls (see pairs())
            if constexpr (Q != 27) {
                if (quads(g)) {
                    const Shape sq = shape_quads(g);
                    if (odd)
                        k_step_aa_odd4<Q><<<sq.grid, sq.block, 0, st>>>(g, cf, VelField<float>{}, a, b, flag);
                    else
                        k_step_aa_even4<Q><<<sq.grid, sq.block, 0, st>>>(g, cf, VelField<float>{}, a, b, flag);
                    return cudaGetLastError();
                }
            }
            if (pairs(g)) {
                const Shape sp = shape_pairs(g, pair_threads<Q>());
                if (odd)
                    k_step_aa_odd2<Q, S><<<sp.grid, sp.block, 0, st>>>(g, cf, VelField<float>{}, a, b, flag);
                else
                    k_step_aa_even2<Q, S, false><<<sp.grid, sp.block, 0, st>>>(g, cf, VelField<float>{}, a, b, flag);
                return cudaGetLastError();
            }
        }
        if (g.link) {
            if (odd)
                k_step_aa<Q, S, true, 1><<<sh.grid, sh.block, 0, st>>>(g, cf, a, b, flag);
            else
                k_step_aa<Q, S, true, 0><<<sh.grid, sh.block, 0, st>>>(g, cf, a, b, flag);
        } else {
            if (odd)
                k_step_aa<Q, S, false, 1><<<sh.grid, sh.block, 0, st>>>(g, cf, a, b, flag);
            else
                k_step_aa<Q, S, false, 0><<<sh.grid, sh.block, 0, st>>>(g, cf, a, b, flag);
        }
        return cudaGetLastError();
    }

    static cudaError_t step_pull_sectors(const Geom& g, const void* coef, const CellList& L, const void* src,
                                         void* dst, int* flag, cudaStream_t st) {
        if (L.count == 0) return cudaSuccess;
        const CF& cf = *static_cast<const CF*>(coef);
        const unsigned long long threads = (unsigned long long)L.count * (32ull / sizeof(ST));  // a sector each
        k_step_pull_sectors<Q, S><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g, cf, L, cpl(src, g), mpl(dst, g),
                                                                                    flag);
        return cudaGetLastError();
    }

    static cudaError_t step_aa_list(const Geom& g, const void* coef, const CellList& L, int odd, const void* src,
                                    void* dst, int* flag, cudaStream_t st) {
        if (L.count == 0) return cudaSuccess;
        const CF& cf = *static_cast<const CF*>(coef);
        const unsigned nb = (L.count + 255) / 256;
        if (odd)
            k_step_aa_list<Q, S, 1><<<nb, 256, 0, st>>>(g, cf, L, cpl(src, g), mpl(dst, g), flag);
        else
            k_step_aa_list<Q, S, 0><<<nb, 256, 0, st>>>(g, cf, L, cpl(src, g), mpl(dst, g), flag);
        return cudaGetLastError();
    }

// Expands to the three layouts times mask / no mask for a kernel template K<Q, S, MASK, LAYOUT>.
#define LBM_BY_LAYOUT(K, ...)                                                                      \
    do {                                                                                           \
        const bool m_ = g.link != nullptr;                                                         \
        if (layout == LAYOUT_PULL) {                                                               \
            if (m_) K<Q, S, true, LAYOUT_PULL><<<sh.grid, sh.block, 0, st>>>(__VA_ARGS__);         \
            else K<Q, S, false, LAYOUT_PULL><<<sh.grid, sh.block, 0, st>>>(__VA_ARGS__);           \
        } else if (layout == LAYOUT_AAODD) {                                                       \
            if (m_) K<Q, S, true, LAYOUT_AAODD><<<sh.grid, sh.block, 0, st>>>(__VA_ARGS__);        \
            else K<Q, S, false, LAYOUT_AAODD><<<sh.grid, sh.block, 0, st>>>(__VA_ARGS__);          \
        } else {                                                                                   \
            if (m_) K<Q, S, true, LAYOUT_LOCAL><<<sh.grid, sh.block, 0, st>>>(__VA_ARGS__);        \
            else K<Q, S, false, LAYOUT_LOCAL><<<sh.grid, sh.block, 0, st>>>(__VA_ARGS__);          \
        }                                                                                          \
    } while (0)

    static cudaError_t moments(const Geom& g, const void* coef, int layout, const void* src, void* rho, void* u,
                               void* Pi, void* f, cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        LBM_BY_LAYOUT(k_moments, g, cf, cpl(src, g), static_cast<T*>(rho), static_cast<T*>(u),
                      static_cast<T*>(Pi), static_cast<T*>(f));
        return cudaGetLastError();
    }

    static cudaError_t totals(const Geom& g, const void* coef, int layout, const void* src, double* part, int* flag,
                              cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        LBM_BY_LAYOUT(k_totals, g, cf, cpl(src, g), part, flag);
        return cudaGetLastError();
    }

    static cudaError_t adj_seed(const Geom& g, const void* coef, int layout, const void* src, const void* grad,
                                void* lam, cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        LBM_BY_LAYOUT(k_adj_seed, g, cf, cpl(src, g), static_cast<const T*>(grad), mfl(lam, g));
        return cudaGetLastError();
    }

    static cudaError_t adj_step(const Geom& g, const void* coef, int layout, const void* src, const void* lam_next,
                                void* lam, double* gpart, cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        if constexpr (S == 3 && Q != 27) {  // FP16 storage without walls: two cells per thread (lbm_adjoint2.cuh;
            // D3Q27 stays one cell per thread: at 128 registers the pair kernel would spill)
            const Shape sp = shape_pairs(g, 128);  // the block shape k_adj_step2 is built for
            if (!g.link && (g.nx % 2) == 0 && sp.nblocks <= sh.nblocks) {  // records fit the per-cell grid's
                const auto a = cpl(src, g);
                const auto ln = cfl(lam_next, g);
                const auto l = mfl(lam, g);
                if (layout == LAYOUT_PULL)
                    k_adj_step2<Q, S, LAYOUT_PULL><<<sp.grid, sp.block, 0, st>>>(g, cf, a, ln, l, gpart);
                else if (layout == LAYOUT_AAODD)
                    k_adj_step2<Q, S, LAYOUT_AAODD><<<sp.grid, sp.block, 0, st>>>(g, cf, a, ln, l, gpart);
                else
                    k_adj_step2<Q, S, LAYOUT_LOCAL><<<sp.grid, sp.block, 0, st>>>(g, cf, a, ln, l, gpart);
                return cudaGetLastError();
            }
        }
        LBM_BY_LAYOUT(k_adj_step, g, cf, cpl(src, g), cfl(lam_next, g), mfl(lam, g), gpart);
        return cudaGetLastError();
    }
#undef LBM_BY_LAYOUT

    static cudaError_t adj_init(const Geom& g, const void* coef, const void* rho0, const void* u0, const void* lam0,
                                void* du0, double* gpart, cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        k_adj_init<Q, T><<<sh.grid, sh.block, 0, st>>>(g, cf, static_cast<const T*>(rho0), static_cast<const T*>(u0),
                                                       cfl(lam0, g), static_cast<T*>(du0), gpart);
        return cudaGetLastError();
    }

    static cudaError_t link_mask(const Geom& g, const uint8_t* solid, uint32_t* link, cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        k_link_mask<Q><<<sh.grid, sh.block, 0, st>>>(g, solid, link);
        return cudaGetLastError();
    }

    static VelField<T> vel_field(const void* u, const Geom& g) {
        VelField<T> v{};
        auto p = static_cast<const T*>(u);
        for (int a = 0; a < Lat<Q>::D; ++a) v.p[a] = p ? p + (size_t)a * g.N : nullptr;
        return v;
    }

    static cudaError_t ade_pull(const Geom& g, const void* coef, const void* u, const void* src, void* dst, int* flag,
                                cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        if constexpr (S == 3) {  // pairs(g) holds for FP16 r-shifted storage only
            if constexpr (Q != 27) {
                if (quads(g)) {
                    const Shape sq = shape_quads(g);
                    k_step_pull4<Q, true><<<sq.grid, sq.block, 0, st>>>(g, cf, vel_field(u, g), cpl(src, g),
                                                                       mpl(dst, g), flag);
                    return cudaGetLastError();
                }
            }
            if (pairs(g)) {
                const Shape sp = shape_pairs(g, pair_threads<Q>());
                k_step_pull2<Q, S, false, true><<<sp.grid, sp.block, 0, st>>>(g, cf, vel_field(u, g), cpl(src, g),
                                                                            mpl(dst, g), flag);
                return cudaGetLastError();
            }
        }
        if (g.link)
            k_ade_pull<Q, S, true><<<sh.grid, sh.block, 0, st>>>(g, cf, vel_field(u, g), cpl(src, g), mpl(dst, g), flag);
        else
            k_ade_pull<Q, S, false><<<sh.grid, sh.block, 0, st>>>(g, cf, vel_field(u, g), cpl(src, g), mpl(dst, g), flag);
        return cudaGetLastError();
    }

    static cudaError_t ade_aa(const Geom& g, const void* coef, const void* u, int odd, const void* src, void* dst,
                              int* flag, cudaStream_t st) {
        const Shape sh = shape_for(g, g.nz - 2 * LBM_SLAB);
        const CF& cf = *static_cast<const CF*>(coef);
        const auto v = vel_field(u, g);
        const auto a = cpl(src, g);
        const auto b = mpl(dst, g);
        if constexpr (S == 3) {  // pairs(g) holds for FP16 r-shifted storage only
            if constexpr (Q != 27) {
                if (quads(g)) {
                    const Shape sq = shape_quads(g);
                    if (odd)
                        k_step_aa_odd4<Q, true><<<sq.grid, sq.block, 0, st>>>(g, cf, v, a, b, flag);
                    else
                        k_step_aa_even4<Q, true><<<sq.grid, sq.block, 0, st>>>(g, cf, v, a, b, flag);
                    return cudaGetLastError();
                }
            }
            if (pairs(g)) {
                const Shape sp = shape_pairs(g, pair_threads<Q>());
                if (odd)
                    k_step_aa_odd2<Q, S, true><<<sp.grid, sp.block, 0, st>>>(g, cf, v, a, b, flag);
                else
                    k_step_aa_even2<Q, S, false, true><<<sp.grid, sp.block, 0, st>>>(g, cf, v, a, b, flag);
                return cudaGetLastError();
            }
        }
        if (g.link) {
            if (odd)
                k_ade_aa<Q, S, true, 1><<<sh.grid, sh.block, 0, st>>>(g, cf, v, a, b, flag);
            else
                k_ade_aa<Q, S, true, 0><<<sh.grid, sh.block, 0, st>>>(g, cf, v, a, b, flag);
        } else {
            if (odd)
                k_ade_aa<Q, S, false, 1><<<sh.grid, sh.block, 0, st>>>(g, cf, v, a, b, flag);
            else
                k_ade_aa<Q, S, false, 0><<<sh.grid, sh.block, 0, st>>>(g, cf, v, a, b, flag);
        }
        return cudaGetLastError();
    }

    static cudaError_t ade_pull_sectors(const Geom& g, const void* coef, const CellList& L, const void* u,
                                        const void* src, void* dst, int* flag, cudaStream_t st) {
        if (L.count == 0) return cudaSuccess;
        const CF& cf = *static_cast<const CF*>(coef);
        const unsigned long long threads = (unsigned long long)L.count * (32ull / sizeof(ST));  // a sector each
        k_ade_pull_sectors<Q, S><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g, cf, L, vel_field(u, g),
                                                                                   cpl(src, g), mpl(dst, g), flag);
        return cudaGetLastError();
    }

    static const Ops& ops() {
        static const Ops o = {&init,     &step_pull, &step_aa,   &step_pull_sectors, &step_aa_list, &moments,
                              &totals,   &adj_seed,  &adj_step,  &adj_init,          &link_mask,    &ade_pull,
                              &ade_aa,   &ade_pull_sectors};
        return o;
    }
};

}  // namespace LBM_VARIANT
}  // namespace lbm
