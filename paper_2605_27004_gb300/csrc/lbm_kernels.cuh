// Device code of the anisotropic-equilibrium BGK lattice Boltzmann library (sm_103a).
//
// Every kernel runs one thread per lattice cell, x fastest, so that each direction's loads and
// stores of a warp touch 32 consecutive elements of one structure-of-arrays plane [q][N]
// (coalesced; the x-1/x+1 shifted reads of a warp straddle one extra 32-byte sector that the
// neighbouring warp reads anyway, and the y/z-shifted rows are re-read from L2). Addresses are a
// per-direction plane pointer plus a 32-bit in-plane offset built from three wrapped x indices
// and nine wrapped row offsets, so a gathered load costs one add and one wide multiply-add.
//
// Arithmetic is carried in the shifted variables d_i = f_i - r_i with r_i the rest equilibrium
// feq_i(rho0, 0; Theta), whatever the storage form: this keeps the FP32 sums of the moments and
// of the relaxation on O(u) quantities instead of O(w_i).
//
// Equilibrium (Eq. 3rd_order_equilibrium with Eq. feq_i; cs2 = 1/3; K~ = Theta - cs2 I):
//   feq_i - r_i = E_i + O_i, evaluated once per opposite pair (i, opp i):
//   even  E_i = drho w_i (1 + 9/2 h_i) + 9/2 rho w_i ((u.c_i)^2 - |u|^2/3)          (= E_opp)
//   odd   O_i = rho [u.c_i w_i (3 + 3 c3 h_i) + w_i c3 ((u.c_i)^3 - |u|^2 u.c_i - 2 c_i.K~.u)]
//                                                                                   (= -O_opp)
//   with drho = rho - rho0, c3 = 9/2 (third order) or 0 (second order).
// BGK relaxation (Eq. LBE_BGK): d_i <- d_i + (feq_i - r_i - d_i)/tau.
//
// FP32 momentum identity: with weights and coefficients rounded to FP32 the discrete first
// moment of the equilibrium is rho u (1 + eps) with a systematic eps ~ 2e-8, which drifts the
// momentum by ~1e-5 over 1000 steps. In exact arithmetic BGK conserves momentum, so the FP32
// storage forms remove the post-collision momentum defect along 3 w_i c_i (a no-op in exact
// arithmetic; mass and the other moments are untouched since sum_i 3 w_i c_i = 0).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_internal.h"
#include "lbm_lattice.cuh"

// Each kernel object is compiled for whole periodic boxes (LBM_SLAB = 0) or for z-slabs
// (LBM_SLAB = 1, the processed planes start at stored plane 1, above the ghost plane). The first
// processed plane is a compile-time constant: read from the kernel parameters it changed the
// register allocation of the FP16 pair kernels and cost them up to 18 % (measured). The two
// builds live in different inline namespaces, so their template instantiations never collide.
#ifndef LBM_SLAB
#define LBM_SLAB 0
#endif
#if LBM_SLAB
#define LBM_VARIANT slab_planes
#else
#define LBM_VARIANT whole_box
#endif

namespace lbm {
inline namespace LBM_VARIANT {

// ---------------------------------------------------------------------------------------------
// Storage forms: 0 FP32 (f), 1 FP64 (f), 2 FP32 shifted (f - r), 3 FP16 shifted (f - r),
// 4 FP16 shifted by the lattice weights (f - w rho0). The arithmetic always runs on d = f - r; the
// forms whose stored value is not d convert with the storage offset Coef::so on load and store.
// ---------------------------------------------------------------------------------------------
template <int S>
struct Store;
template <>
struct Store<0> {
    using type = float;
    using T = float;
    static constexpr bool shifted = false;
    static constexpr bool fix_momentum = true;
    static constexpr bool fold_omega = false;
};
template <>
struct Store<1> {
    using type = double;
    using T = double;
    static constexpr bool shifted = false;
    static constexpr bool fix_momentum = false;
    static constexpr bool fold_omega = false;
};
template <>
struct Store<2> {
    using type = float;
    using T = float;
    static constexpr bool shifted = true;
    static constexpr bool fix_momentum = true;
    static constexpr bool fold_omega = false;
};
template <>
struct Store<3> {
    using type = __half;
    using T = float;
    static constexpr bool shifted = true;
    static constexpr bool fix_momentum = false;  // FP16 rounding (1e-3) dwarfs the 1e-8 bias
    static constexpr bool fold_omega = true;     // see relax()
};
// FP16 storage of f - w rho0, the shift taken literally from the lattice weights: stored values
// carry r_i - w_i rho0 = 9/2 w_i rho0 h_i on top of the O(u) deviation when Theta != cs2 I. It
// exists to measure what the Theta-aware shift of Store<3> gains; one cell per thread only.
template <>
struct Store<4> {
    using type = __half;
    using T = float;
    static constexpr bool shifted = false;
    static constexpr bool fix_momentum = false;
    static constexpr bool fold_omega = true;
};

// read-only (non-coherent) loads: used when the source array is not written by the kernel
__device__ __forceinline__ float ld_ro(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld_ro(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_ro(const __half* p) {
    return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
}
// coherent loads: used by the in-place AA kernels
__device__ __forceinline__ float ld_rw(const float* p) { return *p; }
__device__ __forceinline__ double ld_rw(const double* p) { return *p; }
__device__ __forceinline__ float ld_rw(const __half* p) {
    return __half2float(__ushort_as_half(*reinterpret_cast<const unsigned short*>(p)));
}
__device__ __forceinline__ void st_raw(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_raw(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_raw(__half* p, float v) { *p = __float2half_rn(v); }

template <int S>
__device__ __forceinline__ typename Store<S>::T to_shifted(typename Store<S>::T raw, typename Store<S>::T r) {
    return Store<S>::shifted ? raw : raw - r;
}
template <int S>
__device__ __forceinline__ typename Store<S>::T from_shifted(typename Store<S>::T d, typename Store<S>::T r) {
    return Store<S>::shifted ? d : d + r;
}

// Base pointers of the q planes of a structure-of-arrays buffer, passed by value as a kernel
// parameter so that the bases stay in the constant bank instead of occupying registers.
template <typename P>
struct Planes {
    P* p[27];
};
template <typename P>
Planes<P> planes_of(P* base, int q, uint32_t N) {
    Planes<P> r{};
    for (int i = 0; i < q; ++i) r.p[i] = base ? base + (size_t)i * N : nullptr;
    return r;
}

// ---------------------------------------------------------------------------------------------
// Cell addressing with periodic wrap: X[k] = x - (k - 1), R[a][b] = nx ((y - (a - 1)) +
// ny (z - (b - 1))), all wrapped. Offset of x - c: X[c.x + 1] + R[c.y + 1][c.z + 1];
// offset of x + c: X[1 - c.x] + R[1 - c.y][1 - c.z].
// ---------------------------------------------------------------------------------------------
struct Cell {
    int x, y, z;
    uint32_t n;
    uint32_t N;  // cells per population plane
    uint32_t X[3];
    uint32_t R[3][3];
};

__device__ __forceinline__ bool make_cell(const Geom& g, Cell& c) {
    c.x = blockIdx.x * blockDim.x + threadIdx.x;
    c.y = blockIdx.y * blockDim.y + threadIdx.y;
    c.z = blockIdx.z + LBM_SLAB;
    if (c.x >= g.nx || c.y >= g.ny) return false;
    const uint32_t yy[3] = {(uint32_t)(c.y + 1 == g.ny ? 0 : c.y + 1), (uint32_t)c.y,
                            (uint32_t)(c.y == 0 ? g.ny - 1 : c.y - 1)};
    const uint32_t zz[3] = {(uint32_t)(c.z + 1 == g.nz ? 0 : c.z + 1), (uint32_t)c.z,
                            (uint32_t)(c.z == 0 ? g.nz - 1 : c.z - 1)};
    c.X[0] = c.x + 1 == g.nx ? 0u : (uint32_t)(c.x + 1);
    c.X[1] = (uint32_t)c.x;
    c.X[2] = c.x == 0 ? (uint32_t)(g.nx - 1) : (uint32_t)(c.x - 1);
    const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) c.R[a][b] = nx * (yy[a] + ny * zz[b]);
    c.n = c.X[1] + c.R[1][1];
    c.N = g.N;
    return true;
}

__device__ __forceinline__ uint32_t off_minus(const Cell& c, Vec3 v) { return c.X[v.x + 1] + c.R[v.y + 1][v.z + 1]; }
__device__ __forceinline__ uint32_t off_plus(const Cell& c, Vec3 v) { return c.X[1 - v.x] + c.R[1 - v.y][1 - v.z]; }

template <bool MASK>
__device__ __forceinline__ uint32_t link_of(const Geom& g, const Cell& c) {
    return MASK ? __ldg(g.link + c.n) : 0u;
}
__device__ __forceinline__ bool link_bit(uint32_t lw, int i) { return (lw >> i) & 1u; }

// Gather of the pre-collision populations of one cell in shifted form (see Layout).
template <int Q, int S, bool MASK, int LAYOUT, bool RO>
__device__ __forceinline__ void gather(const Cell& c, uint32_t lw, const Coef<typename Store<S>::T>& cf,
                                       const Planes<const typename Store<S>::type>& src,
                                       typename Store<S>::T (&d)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const Vec3 v = vel<Q>(i);
        const typename Store<S>::type* p;
        if (LAYOUT == LAYOUT_LOCAL || i == 0) {
            p = src.p[i] + c.n;
        } else {
            const int slot_n = LAYOUT == LAYOUT_PULL ? i : opp(i);  // slot read from the neighbour
            const int slot_w = LAYOUT == LAYOUT_PULL ? opp(i) : i;  // slot read on a wall link
            if (MASK) {
                // Both candidates as 32-bit offsets from the lower plane of the pair (i, opp i), so
                // that the wall select is one select of an offset instead of a 64-bit address
                // (measured on the porous D3Q27 box: FP16 pull 0.406 -> 0.431 of the copy peak).
                // Offsets stay below 2N < 2^32.
                const int lo = slot_n < slot_w ? slot_n : slot_w;
                const uint32_t offn = off_minus(c, v) + (slot_n > lo ? c.N : 0u);
                const uint32_t offw = c.n + (slot_w > lo ? c.N : 0u);
                p = src.p[lo] + (link_bit(lw, i) ? offw : offn);
            } else {
                p = src.p[slot_n] + off_minus(c, v);
            }
        }
        const auto raw = RO ? ld_ro(p) : ld_rw(p);
        d[i] = to_shifted<S>(raw, cf.so[i]);
    }
}

// ---------------------------------------------------------------------------------------------
// Moments and equilibrium
// ---------------------------------------------------------------------------------------------
template <typename T>
struct Macro {
    T drho, rho, jx, jy, jz, ux, uy, uz;
};

template <typename T>
__device__ __forceinline__ void add_c(Vec3 v, T val, T& x, T& y, T& z) {
    if (v.x == 1) x += val;
    if (v.x == -1) x -= val;
    if (v.y == 1) y += val;
    if (v.y == -1) y -= val;
    if (v.z == 1) z += val;
    if (v.z == -1) z -= val;
}

template <int Q, typename T>
__device__ __forceinline__ Macro<T> macro_of(const T (&d)[Q], T rho0) {
    T s = d[0], jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int k = 0; k < Lat<Q>::P; ++k) {
        const T a = d[2 * k + 1], b = d[2 * k + 2];
        s += a + b;
        add_c<T>(vel<Q>(2 * k + 1), a - b, jx, jy, jz);
    }
    Macro<T> m;
    m.drho = s;
    m.rho = rho0 + s;
    m.jx = jx;
    m.jy = jy;
    m.jz = jz;
    const T inv = T(1) / m.rho;
    m.ux = jx * inv;
    m.uy = jy * inv;
    m.uz = Lat<Q>::D == 3 ? jz * inv : T(0);
    return m;
}

// v . (ax, ay, az) for a lattice vector with components in {-1, 0, 1}
template <typename T>
__device__ __forceinline__ T vdot(Vec3 v, T ax, T ay, T az) {
    T r = T(0);
    if (v.x == 1) r += ax;
    if (v.x == -1) r -= ax;
    if (v.y == 1) r += ay;
    if (v.y == -1) r -= ay;
    if (v.z == 1) r += az;
    if (v.z == -1) r -= az;
    return r;
}

// Per-cell invariants of the equilibrium.
template <typename T>
struct EqCell {
    T drho, rho, ux, uy, uz, usq, kx, ky, kz, r45;
};

template <typename T>
__device__ __forceinline__ EqCell<T> eq_cell(const Coef<T>& cf, T drho, T rho, T ux, T uy, T uz) {
    EqCell<T> e;
    e.drho = drho;
    e.rho = rho;
    e.ux = ux;
    e.uy = uy;
    e.uz = uz;
    e.usq = ux * ux + uy * uy + uz * uz;
    e.kx = cf.K[0] * ux + cf.K[3] * uy + cf.K[4] * uz;
    e.ky = cf.K[3] * ux + cf.K[1] * uy + cf.K[5] * uz;
    e.kz = cf.K[4] * ux + cf.K[5] * uy + cf.K[2] * uz;
    e.r45 = T(4.5) * rho;
    return e;
}

// Even and odd parts of feq - r for the direction pair (i, opp i), i = 2k + 1.
template <int Q, typename T>
__device__ __forceinline__ void pair_eq(const Coef<T>& cf, const EqCell<T>& e, int k, T& E, T& O, T& uc) {
    const int i = 2 * k + 1;
    const Vec3 v = vel<Q>(i);
    const T w = T(weight<Q>(i));
    uc = vdot<T>(v, e.ux, e.uy, e.uz);
    const T qk = vdot<T>(v, e.kx, e.ky, e.kz);
    E = e.drho * cf.A[i] + w * e.r45 * (uc * uc - e.usq * T(1.0 / 3.0));
    O = e.rho * (uc * cf.B[i] + w * cf.c3 * (uc * (uc * uc - e.usq) - T(2) * qk));
}

template <int Q, typename T>
__device__ __forceinline__ T rest_eq(const Coef<T>& cf, const EqCell<T>& e) {
    return e.drho * cf.A[0] - T(weight<Q>(0)) * e.r45 * e.usq * T(1.0 / 3.0);
}

// d_i <- (1 - 1/tau) d_i + (feq_i - r_i)/tau for the equilibrium state e (Eq. LBE_BGK).
// FOLD evaluates the same expression with 1/tau folded into the per-cell factors (om drho,
// om rho, om 4.5 rho) and 2 K~.u precomputed, which shortens the dependency chain of every
// population; it is used where the kernel is instruction-bound (FP16 storage; measured D3Q27
// FP16 0.66 -> 0.70 of the copy peak) and rounds differently in the last bits.
template <int Q, typename T, bool FOLD = false>
__device__ __forceinline__ void relax(const Coef<T>& cf, const EqCell<T>& e, T (&d)[Q]) {
    const T om = cf.omega, om1 = T(1) - cf.omega;
    if (FOLD) {
        const T omdrho = om * e.drho, omrho = om * e.rho, omr45 = om * e.r45;
        const T kx2 = T(2) * e.kx, ky2 = T(2) * e.ky, kz2 = T(2) * e.kz;
        const T usq3 = e.usq * T(1.0 / 3.0);
        d[0] = om1 * d[0] + (omdrho * cf.A[0] - T(weight<Q>(0)) * omr45 * usq3);
#pragma unroll
        for (int k = 0; k < Lat<Q>::P; ++k) {
            const int i = 2 * k + 1;
            const Vec3 v = vel<Q>(i);
            const T w = T(weight<Q>(i));
            const T uc = vdot<T>(v, e.ux, e.uy, e.uz);
            const T qk2 = vdot<T>(v, kx2, ky2, kz2);
            const T E = omdrho * cf.A[i] + (w * omr45) * (uc * uc - usq3);
            const T O = omrho * (uc * cf.B[i] + (w * cf.c3) * (uc * (uc * uc - e.usq) - qk2));
            d[i] = om1 * d[i] + (E + O);
            d[i + 1] = om1 * d[i + 1] + (E - O);
        }
        return;
    }
    d[0] = om1 * d[0] + om * rest_eq<Q, T>(cf, e);
#pragma unroll
    for (int k = 0; k < Lat<Q>::P; ++k) {
        T E, O, uc;
        pair_eq<Q, T>(cf, e, k, E, O, uc);
        d[2 * k + 1] = om1 * d[2 * k + 1] + om * (E + O);
        d[2 * k + 2] = om1 * d[2 * k + 2] + om * (E - O);
    }
}

// BGK collision in place on shifted populations; returns the macroscopic state.
template <int Q, typename T, bool FIX, bool FOLD = false>
__device__ __forceinline__ Macro<T> bgk(const Coef<T>& cf, T (&d)[Q]) {
    const Macro<T> m = macro_of<Q, T>(d, cf.rho0);
    const EqCell<T> e = eq_cell<T>(cf, m.drho, m.rho, m.ux, m.uy, m.uz);
    relax<Q, T, FOLD>(cf, e, d);
    if (FIX) {
        // post-collision momentum defect, removed along 3 w_i c_i
        T ex = -m.jx, ey = -m.jy, ez = -m.jz;
#pragma unroll
        for (int k = 0; k < Lat<Q>::P; ++k) add_c<T>(vel<Q>(2 * k + 1), d[2 * k + 1] - d[2 * k + 2], ex, ey, ez);
#pragma unroll
        for (int k = 0; k < Lat<Q>::P; ++k) {
            const Vec3 v = vel<Q>(2 * k + 1);
            const T corr = T(3.0 * weight<Q>(2 * k + 1)) * vdot<T>(v, ex, ey, ez);
            d[2 * k + 1] -= corr;
            d[2 * k + 2] += corr;
        }
    }
    return m;
}

template <typename T>
__device__ __forceinline__ bool bad_cell(const Macro<T>& m) {
    return !(m.rho > T(0)) || !isfinite(m.ux + m.uy + m.uz);
}

// With walls, whether this lane stores: the lanes of a warp that share one 32-byte sector of a
// population plane (8 FP32, 16 FP16, 4 FP64 cells) store when any of them is fluid; a solid lane
// among them stores zeros into its own never-read slots, so the sector is written whole (a
// partly written sector is read from DRAM and merged before write-back), and sectors of solid
// cells only are not written at all (measured on the porous D3Q27 box: FP32 0.66 -> 0.69).
template <typename E>
__device__ __forceinline__ bool store_group(unsigned act, bool solid) {
    constexpr int G = 32 / (int)sizeof(E);
    const unsigned fl = __ballot_sync(act, !solid);
    const int lane = (threadIdx.x + threadIdx.y * blockDim.x) & 31;
    const unsigned gm = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    return (fl & gm) != 0u;
}

// ---------------------------------------------------------------------------------------------
// Fused stream + collide, two arrays, pull form: gather f(t) from the post-collision array of
// the previous step, relax, store at the own cell. One launch per time step.
// ---------------------------------------------------------------------------------------------
template <int Q, int S, bool MASK>
__global__ void __launch_bounds__(256) k_step_pull(Geom g, Coef<typename Store<S>::T> cf,
                                                   const Planes<const typename Store<S>::type> src,
                                                   const Planes<typename Store<S>::type> dst, int* __restrict__ flag) {
    using T = typename Store<S>::T;
    Cell c;
    if (!make_cell(g, c)) return;
    const uint32_t lw = link_of<MASK>(g, c);
    // With walls, a solid cell's slots are never read (a gather that meets a solid neighbour takes
    // the own cell's opposite slot) nor written by another cell, so a solid lane may store zeros
    // there in the same store instructions as the fluid lanes of its sector (store_group).
    const bool solid = MASK && (lw & LINK_SOLID);
    const unsigned act = __activemask();
    if (MASK && __all_sync(act, solid)) return;
    T d[Q];
    if (MASK && __all_sync(act, lw == 0u)) {
        // no lane of the warp has a wall link: the branch-free gather (in the porous medium of
        // overlapping spheres about 28 % of the warps, 40 % of the fluid cells)
        gather<Q, S, false, LAYOUT_PULL, true>(c, 0u, cf, src, d);
    } else if (!solid) {
        gather<Q, S, MASK, LAYOUT_PULL, true>(c, lw, cf, src, d);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = T(0);
    }
    const Macro<T> m = bgk<Q, T, Store<S>::fix_momentum, Store<S>::fold_omega>(cf, d);
    if (!solid && bad_cell(m)) *flag = 1;
    if (MASK && !store_group<typename Store<S>::type>(act, solid)) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) st_raw(dst.p[i] + c.n, solid ? T(0) : from_shifted<S>(d[i], cf.so[i]));
}

// ---------------------------------------------------------------------------------------------
// AA pattern (one array, in place; src == dst allowed).
//   even: read A[i][x], write f*_i to A[opp i][x]                     (state LOCAL -> AAODD)
//   odd:  read f_i per AAODD, write f*_i to A[i][x + c_i], or to A[opp i][x] if x + c_i is
//         solid                                                         (state AAODD -> LOCAL)
// Each thread writes exactly the slots it read, so the in-place update is race free. The link
// bit of x + c_i is the bit of direction opp(i).
// ---------------------------------------------------------------------------------------------
template <int Q, int S, bool MASK, int ODD>
__device__ __forceinline__ void aa_store(const Cell& c, uint32_t lw, const Coef<typename Store<S>::T>& cf,
                                         const Planes<typename Store<S>::type>& dst,
                                         const typename Store<S>::T (&d)[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        typename Store<S>::type* p;
        if (i == 0) {
            p = dst.p[0] + c.n;
        } else if (!ODD) {
            p = dst.p[opp(i)] + c.n;
        } else {
            const Vec3 v = vel<Q>(i);
            if (MASK && link_bit(lw, opp(i)))
                p = dst.p[opp(i)] + c.n;
            else
                p = dst.p[i] + off_plus(c, v);
        }
        st_raw(p, from_shifted<S>(d[i], cf.so[i]));
    }
}

template <int Q, int S, bool MASK, int ODD>
__global__ void __launch_bounds__(256) k_step_aa(Geom g, Coef<typename Store<S>::T> cf,
                                                 const Planes<const typename Store<S>::type> src,
                                                 const Planes<typename Store<S>::type> dst, int* __restrict__ flag) {
    using T = typename Store<S>::T;
    Cell c;
    if (!make_cell(g, c)) return;
    const uint32_t lw = link_of<MASK>(g, c);
    if (MASK && (lw & LINK_SOLID)) return;
    T d[Q];
    // a cell without wall links needs no selects; taken warp-wide so that lanes do not diverge
    const bool clean = MASK && __all_sync(__activemask(), lw == 0u);
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
    const Macro<T> m = bgk<Q, T, Store<S>::fix_momentum, Store<S>::fold_omega>(cf, d);
    if (bad_cell(m)) *flag = 1;
    if (clean)
        aa_store<Q, S, false, ODD>(c, 0u, cf, dst, d);
    else
        aa_store<Q, S, MASK, ODD>(c, lw, cf, dst, d);
}

// ---------------------------------------------------------------------------------------------
// AA steps over the fluid-cell list (CellList): one fluid cell per thread, no solid lanes. Used for
// FP16 storage with walls, where the one-cell kernels are limited by issued instructions and the
// solid lanes of mixed warps (about 30 % of the lanes in the porous medium) issue them too
// (porous D3Q27 512^3: 0.465 -> 0.483 of the copy peak on fluid accounting). The in-place AA
// kernels store fluid slots only anyway; for the pull scheme a fluid-cell list loses the
// whole-sector stores of the grid kernel (measured 0.443 -> 0.384), so the pull step runs over
// 16-cell sectors instead (k_step_pull_sectors). Four blocks per SM (64 registers; the odd step
// had taken 77, three blocks): 0.483 -> 0.490.
// ---------------------------------------------------------------------------------------------
// Cell n of the list's box, its coordinates from the exact reciprocals of nx and nx ny.
__device__ __forceinline__ void make_cell_index(const Geom& g, const CellList& L, uint32_t n, Cell& c) {
    const uint32_t z = (uint32_t)__umul64hi((unsigned long long)n, L.rnxy);
    const uint32_t r = n - z * ((uint32_t)g.nx * (uint32_t)g.ny);
    const uint32_t y = (uint32_t)__umul64hi((unsigned long long)r, L.rnx);
    c.x = (int)(r - y * (uint32_t)g.nx);
    c.y = (int)y;
    c.z = (int)z;
    const uint32_t yy[3] = {(uint32_t)(c.y + 1 == g.ny ? 0 : c.y + 1), (uint32_t)c.y,
                            (uint32_t)(c.y == 0 ? g.ny - 1 : c.y - 1)};
    const uint32_t zz[3] = {(uint32_t)(c.z + 1 == g.nz ? 0 : c.z + 1), (uint32_t)c.z,
                            (uint32_t)(c.z == 0 ? g.nz - 1 : c.z - 1)};
    c.X[0] = c.x + 1 == g.nx ? 0u : (uint32_t)(c.x + 1);
    c.X[1] = (uint32_t)c.x;
    c.X[2] = c.x == 0 ? (uint32_t)(g.nx - 1) : (uint32_t)(c.x - 1);
    const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) c.R[a][b] = nx * (yy[a] + ny * zz[b]);
    c.n = n;
    c.N = g.N;
}

__device__ __forceinline__ bool make_cell_list(const Geom& g, const CellList& L, Cell& c) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.count) return false;
    make_cell_index(g, L, __ldg(L.idx + t), c);
    return true;
}

// Pull step over the list of 32-byte sectors (16 FP16 or 8 FP32 cells of a plane) that hold a
// fluid cell: G consecutive lanes take one sector, so a warp never spends lanes on sectors of solid
// cells only (11 % of the FP16 sectors of the porous medium, against 2 % of whole solid warps in
// the grid kernel), and its stores stay whole sectors as in k_step_pull (solid lanes store zeros
// into their never-read slots). Lanes past the processed planes (the ends of the list) load and
// store nothing. Ordering the list so that sectors without wall links come first in each window
// of 32 (more warps on the branch-free gather) measured +0.25 % and is not done.
template <int Q, int S>
__global__ void __launch_bounds__(256) k_step_pull_sectors(Geom g, Coef<typename Store<S>::T> cf, CellList L,
                                                           const Planes<const typename Store<S>::type> src,
                                                           const Planes<typename Store<S>::type> dst,
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
    const Macro<T> m = bgk<Q, T, Store<S>::fix_momentum, Store<S>::fold_omega>(cf, d);
    if (!solid && bad_cell(m)) *flag = 1;
    const bool store = store_group<typename Store<S>::type>(act, solid);
    if (!valid || !store) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) st_raw(dst.p[i] + c.n, solid ? T(0) : from_shifted<S>(d[i], cf.so[i]));
}

template <int Q, int S, int ODD>
__global__ void __launch_bounds__(256, 4) k_step_aa_list(Geom g, Coef<typename Store<S>::T> cf, CellList L,
                                                      const Planes<const typename Store<S>::type> src,
                                                      const Planes<typename Store<S>::type> dst,
                                                      int* __restrict__ flag) {
    using T = typename Store<S>::T;
    Cell c;
    if (!make_cell_list(g, L, c)) return;
    const uint32_t lw = __ldg(g.link + c.n);
    T d[Q];
    const bool clean = __all_sync(__activemask(), lw == 0u);
    if (clean) {
        if (ODD)
            gather<Q, S, false, LAYOUT_AAODD, false>(c, 0u, cf, src, d);
        else
            gather<Q, S, false, LAYOUT_LOCAL, false>(c, 0u, cf, src, d);
    } else if (ODD) {
        gather<Q, S, true, LAYOUT_AAODD, false>(c, lw, cf, src, d);
    } else {
        gather<Q, S, true, LAYOUT_LOCAL, false>(c, lw, cf, src, d);
    }
    const Macro<T> m = bgk<Q, T, Store<S>::fix_momentum, Store<S>::fold_omega>(cf, d);
    if (bad_cell(m)) *flag = 1;
    if (clean)
        aa_store<Q, S, false, ODD>(c, 0u, cf, dst, d);
    else
        aa_store<Q, S, true, ODD>(c, lw, cf, dst, d);
}

// ---------------------------------------------------------------------------------------------
// Initial state f(0) = feq(rho, u), written so that the chosen layout gathers it back.
// ---------------------------------------------------------------------------------------------
template <int Q, int S, bool MASK, int LAYOUT>
__global__ void __launch_bounds__(256) k_init(Geom g, Coef<typename Store<S>::T> cf,
                                              const typename Store<S>::T* __restrict__ rho_in,
                                              const typename Store<S>::T* __restrict__ u_in,
                                              const Planes<typename Store<S>::type> dst) {
    using T = typename Store<S>::T;
    Cell c;
    if (!make_cell(g, c)) return;
    const uint32_t lw = link_of<MASK>(g, c);
    if (MASK && (lw & LINK_SOLID)) return;
    const uint32_t N = g.N;
    const T rho = rho_in ? rho_in[c.n] : cf.rho0;
    const T ux = u_in ? u_in[c.n] : T(0);
    const T uy = u_in ? u_in[N + c.n] : T(0);
    const T uz = (u_in && Lat<Q>::D == 3) ? u_in[2 * (size_t)N + c.n] : T(0);
    const EqCell<T> e = eq_cell<T>(cf, rho - cf.rho0, rho, ux, uy, uz);
    T d[Q];
    d[0] = rest_eq<Q, T>(cf, e);
#pragma unroll
    for (int k = 0; k < Lat<Q>::P; ++k) {
        T E, O, uc;
        pair_eq<Q, T>(cf, e, k, E, O, uc);
        d[2 * k + 1] = E + O;
        d[2 * k + 2] = E - O;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        typename Store<S>::type* p;
        if (LAYOUT == LAYOUT_LOCAL || i == 0) {
            p = dst.p[i] + c.n;
        } else {
            // the slot the PULL gather reads f_i(x) from
            if (MASK && link_bit(lw, i))
                p = dst.p[opp(i)] + c.n;
            else
                p = dst.p[i] + off_minus(c, vel<Q>(i));
        }
        st_raw(p, from_shifted<S>(d[i], cf.so[i]));
    }
}

// ---------------------------------------------------------------------------------------------
// Link words from a byte mask: bit i = solid(x - c_i), bit 31 = solid(x).
// ---------------------------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(256) k_link_mask(Geom g, const uint8_t* __restrict__ solid,
                                                   uint32_t* __restrict__ link) {
    Cell c;
    if (!make_cell(g, c)) return;
    uint32_t lw = solid[c.n] ? LINK_SOLID : 0u;
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (solid[off_minus(c, vel<Q>(i))]) lw |= 1u << i;
    link[c.n] = lw;
}

// ---------------------------------------------------------------------------------------------
// Observables of f(t): rho, u, Pi (Eqs. a0discrete_f, a1discrete_f; Appendix E second moment),
// and optionally the unshifted populations f_i in direction order.
// ---------------------------------------------------------------------------------------------
__host__ __device__ constexpr int pi_a(int D, int k) {
    return D == 2 ? (k == 0 ? 0 : k == 1 ? 1 : 0) : (k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 2 : k == 3 ? 0 : k == 4 ? 0 : 1);
}
__host__ __device__ constexpr int pi_b(int D, int k) {
    return D == 2 ? (k == 0 ? 0 : k == 1 ? 1 : 1) : (k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 2 : k == 3 ? 1 : k == 4 ? 2 : 2);
}
// index into the xx, yy, zz, xy, xz, yz ordering of Coef::Pirest
__host__ __device__ constexpr int pi_full(int D, int k) { return D == 2 ? (k == 2 ? 3 : k) : k; }
__host__ __device__ constexpr int comp(Vec3 v, int a) { return a == 0 ? v.x : a == 1 ? v.y : v.z; }

template <int Q, int S, bool MASK, int LAYOUT>
__global__ void __launch_bounds__(256) k_moments(Geom g, Coef<typename Store<S>::T> cf,
                                                 const Planes<const typename Store<S>::type> src,
                                                 typename Store<S>::T* __restrict__ rho_out,
                                                 typename Store<S>::T* __restrict__ u_out,
                                                 typename Store<S>::T* __restrict__ pi_out,
                                                 typename Store<S>::T* __restrict__ f_out) {
    using T = typename Store<S>::T;
    constexpr int D = Lat<Q>::D;
    constexpr int NP = D == 2 ? 3 : 6;
    Cell c;
    if (!make_cell(g, c)) return;
    const size_t N = g.N;
    const uint32_t lw = link_of<MASK>(g, c);
    if (MASK && (lw & LINK_SOLID)) {
        if (rho_out) rho_out[c.n] = T(0);
        if (u_out)
            for (int a = 0; a < D; ++a) u_out[a * N + c.n] = T(0);
        if (pi_out)
            for (int k = 0; k < NP; ++k) pi_out[k * N + c.n] = T(0);
        if (f_out)
            for (int i = 0; i < Q; ++i) f_out[i * N + c.n] = T(0);
        return;
    }
    T d[Q];
    gather<Q, S, MASK, LAYOUT, true>(c, lw, cf, src, d);
    const Macro<T> m = macro_of<Q, T>(d, cf.rho0);
    if (rho_out) rho_out[c.n] = m.rho;
    if (u_out) {
        u_out[c.n] = m.ux;
        u_out[N + c.n] = m.uy;
        if (D == 3) u_out[2 * N + c.n] = m.uz;
    }
    if (pi_out) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            T s = T(0);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int p = comp(vel<Q>(i), pi_a(D, k)) * comp(vel<Q>(i), pi_b(D, k));
                if (p == 1) s += d[i];
                if (p == -1) s -= d[i];
            }
            pi_out[k * N + c.n] = cf.Pirest[pi_full(D, k)] + s;
        }
    }
    if (f_out) {
#pragma unroll
        for (int i = 0; i < Q; ++i) f_out[i * N + c.n] = d[i] + cf.r[i];
    }
}

// ---------------------------------------------------------------------------------------------
// Block reductions: FP64 throughout for totals; for gradient records the 32 lanes of a warp are
// summed in the arithmetic type first, then the warps and all later accumulation are FP64.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ long long block_linear() {
    return (long long)blockIdx.x + (long long)gridDim.x * ((long long)blockIdx.y + (long long)gridDim.y * blockIdx.z);
}

// Block sum of W values per thread. The 32 lanes of a warp are added in the value type T; then
// thread k < W adds component k of the (at most 8) warp sums in FP64, in parallel. Returns the
// block sum of component tid for threads tid < W (0 for the others).
template <int W, typename T>
__device__ __forceinline__ double block_sum_lane(T (&v)[W]) {
    __shared__ T sh[8][W];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        T s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    double s = 0.0;
    if (tid < W)
        for (int w = 0; w < nwarps; ++w) s += (double)sh[w][tid];
    return s;
}

// Totals over fluid cells: partial[block][0] = sum rho, [1..3] = sum j, in FP64.
template <int Q, int S, bool MASK, int LAYOUT>
__global__ void __launch_bounds__(256) k_totals(Geom g, Coef<typename Store<S>::T> cf,
                                                const Planes<const typename Store<S>::type> src,
                                                double* __restrict__ partials, int* __restrict__ flag) {
    using T = typename Store<S>::T;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    Cell c;
    if (make_cell(g, c)) {
        const uint32_t lw = link_of<MASK>(g, c);
        if (!(MASK && (lw & LINK_SOLID))) {
            T d[Q];
            gather<Q, S, MASK, LAYOUT, true>(c, lw, cf, src, d);
            const Macro<T> m = macro_of<Q, T>(d, cf.rho0);
            if (bad_cell(m)) *flag = 1;
            v[0] = (double)m.rho;
            v[1] = (double)m.jx;
            v[2] = (double)m.jy;
            v[3] = (double)m.jz;
        }
    }
    const double s = block_sum_lane<4, double>(v);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid < 4) partials[block_linear() * 4 + tid] = s;
}

// ---------------------------------------------------------------------------------------------
// Discrete adjoint. lambda_t,i(x) = dL/df_i(x, t) for the pre-collision state, plain [q][N].
//   seed   lambda_T,i = sum_a g_a (c_ia - u_a) / rho                               (du/df)
//   step   mu_i(x) = lambda_{t+1,i}(x + c_i), or lambda_{t+1,opp i}(x) if x + c_i is solid
//          (transpose of streaming with bounce-back), then
//          lambda_t,i = (1 - 1/tau) mu_i + (1/tau) (v0 + c_i . v)                 (J_C^T mu)
//          with v0 = sum_i mu_i dfeq_i/drho |_j and v = sum_i mu_i dfeq_i/dj.
//   params dL/dtau  += -(1/tau^2) sum_i mu_i (feq_i - f_i)
//          dL/dK~ab += (1/tau) sum_i mu_i dfeq_i/dK~ab (and once more at t = 0 through f(0) =
//          feq(rho0, u0), without the 1/tau).
// With feq_i = w_i rho P_i(u), u = j/rho, and P_i the bracket of the equilibrium:
//   dP_i/du = c_i (3 + 9 uc + c3 (3 uc^2 - |u|^2 + 3 h_i)) - u (3 + 2 c3 uc) - 2 c3 K~ c_i
//   P_i - u.dP_i/du = 1 + 9/2 h_i - 9/2 uc^2 + 3/2 |u|^2 - 2 c3 uc (uc^2 - |u|^2)
//   dfeq_i/dK~ab = w_i rho [9/2 (c_a c_b - d_ab/3) + c3 (3 uc (c_a c_b - d_ab/3) - 2 c_a u_b)]
// The per-pair sums below use mu_i + mu_opp (even terms) and mu_i - mu_opp (odd terms).
// ---------------------------------------------------------------------------------------------
template <typename T>
struct AdjAcc {
    T v0, B, P0, Q0, gE;  // gE = sum_i mu_i (feq_i - f_i) when the populations are given
    T Va[3], V[3];
    T P[6], Qm[6];  // xx yy zz xy xz yz
};

// Component index of the symmetric pair (a, b) in the xx yy zz xy xz yz order, and of the
// symmetric triple (a, b, c) among the third-order components xxy xxz xyy yyz xzz yzz xyz
// (a triple with one index three times, e.g. xxx, equals the first moment on the lattice,
// since c_a^3 = c_a for components in {-1, 0, 1}).
__host__ __device__ constexpr int sym2(int a, int b) {
    return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5));
}
__host__ __device__ constexpr int sym3_sorted(int a, int b, int c) {
    return (a == 0 && b == 0 && c == 1) ? 0 : (a == 0 && b == 0 && c == 2) ? 1 : (a == 0 && b == 1 && c == 1) ? 2
           : (a == 1 && b == 1 && c == 2) ? 3 : (a == 0 && b == 2 && c == 2) ? 4 : (a == 1 && b == 2 && c == 2) ? 5 : 6;
}
__host__ __device__ constexpr int sym3(int a, int b, int c) {
    // lo <= mid <= hi, then the sorted triple's position in the list above
    return sym3_sorted(a < b ? (a < c ? a : c) : (b < c ? b : c),
                       a + b + c - (a < b ? (a < c ? a : c) : (b < c ? b : c)) - (a > b ? (a > c ? a : c) : (b > c ? b : c)),
                       a > b ? (a > c ? a : c) : (b > c ? b : c));
}

// The per-pair sums of the adjoint through the moments of mu (even part sm = w (mu_i + mu_opp),
// odd part dm = w (mu_i - mu_opp)): S0 = sum w mu, S2_ab = sum sm c_a c_b, D1_a = sum dm c_a,
// D3_abc = sum dm c_a c_b c_c. Every sum the transposed Jacobian needs is a polynomial in u and
// K~ times these (h_i = c_i.K~.c_i + h_0, h_0 = -cs2 tr K~):
//   Q0 = u.D1,  B = 3 S0 + 2 c3 Q0,  P_ab = S2_ab,  Qm_ab = D3_abc u_c,  V = D1,
//   v0 = (1 + 3/2 |u|^2) S0 + 9/2 (K~:S2 + h_0 S0) - 9/2 u.S2.u - 2 c3 (D3[u,u,u] - |u|^2 Q0),
//   Va_a = 3 D1_a + 9 (S2 u)_a + c3 (3 D3[a,u,u] - |u|^2 D1_a + 3 (K~_bc D3_abc + h_0 D1_a)),
// i.e. the direction loop only adds mu into 16 (D3Q19, D2Q9) or 17 (D3Q27) moments. The
// tau-gradient sum gE = sum_i mu_i (feq_i - f_i) keeps its per-direction differences (each
// difference of two close values is exact, so the non-equilibrium part keeps its precision).
template <int Q, typename T>
__device__ __forceinline__ AdjAcc<T> adj_accumulate(const Coef<T>& cf, const EqCell<T>& e, const T (&mu)[Q],
                                                    const T* d) {
    constexpr int D = Lat<Q>::D;
    T S0 = T(weight<Q>(0)) * mu[0], S2[6], D1[3], D3[7], gE = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) S2[k] = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) D1[a] = T(0);
#pragma unroll
    for (int k = 0; k < 7; ++k) D3[k] = T(0);
    if (d) gE = mu[0] * (rest_eq<Q, T>(cf, e) - d[0]);
#pragma unroll
    for (int k = 0; k < Lat<Q>::P; ++k) {
        const int i = 2 * k + 1;
        const Vec3 v = vel<Q>(i);
        const int c[3] = {v.x, v.y, v.z};
        const T w = T(weight<Q>(i));
        const T sm = w * (mu[i] + mu[i + 1]), dm = w * (mu[i] - mu[i + 1]);
        if (d) {
            T E, O, uc;
            pair_eq<Q, T>(cf, e, k, E, O, uc);
            gE += mu[i] * ((E + O) - d[i]) + mu[i + 1] * ((E - O) - d[i + 1]);
        }
        S0 += sm;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (c[a] == 1) D1[a] += dm;
            if (c[a] == -1) D1[a] -= dm;
#pragma unroll
            for (int b = a; b < 3; ++b) {
                const int p2 = c[a] * c[b];
                if (p2 == 1) S2[sym2(a, b)] += sm;
                if (p2 == -1) S2[sym2(a, b)] -= sm;
#pragma unroll
                for (int cc = b; cc < 3; ++cc) {
                    if (a == b && b == cc) continue;  // c_a^3 = c_a: part of D1
                    const int p3 = c[a] * c[b] * c[cc];
                    if (p3 == 1) D3[sym3(a, b, cc)] += dm;
                    if (p3 == -1) D3[sym3(a, b, cc)] -= dm;
                }
            }
        }
    }
    const T u[3] = {e.ux, e.uy, e.uz};
    const T usq = e.usq, c3 = cf.c3, h0 = cf.h[0];
    AdjAcc<T> A;
    A.P0 = S0;
    A.Q0 = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) A.Q0 += u[a] * D1[a];
    A.B = T(3) * S0 + T(2) * c3 * A.Q0;
    A.gE = gE;
    T S2u[3], D3uu[3], KD3[3];
    T uS2u = T(0), KS2 = T(0), D3uuu = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        S2u[a] = D3uu[a] = KD3[a] = T(0);
        A.V[a] = D1[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
#pragma unroll
        for (int b = 0; b < D; ++b) {
            S2u[a] += S2[sym2(a, b)] * u[b];
            KS2 += cf.K[sym2(a, b)] * S2[sym2(a, b)];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                D3uu[a] += ((a == b && b == c) ? D1[a] : D3[sym3(a, b, c)]) * (u[b] * u[c]);
                KD3[a] += cf.K[sym2(b, c)] * ((a == b && b == c) ? D1[a] : D3[sym3(a, b, c)]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        uS2u += u[a] * S2u[a];
        D3uuu += u[a] * D3uu[a];
    }
    A.v0 = (T(1) + T(1.5) * usq) * S0 + T(4.5) * (KS2 + h0 * S0) - T(4.5) * uS2u -
           T(2) * c3 * (D3uuu - usq * A.Q0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        A.Va[a] = T(3) * D1[a] + T(9) * S2u[a] +
                  c3 * (T(3) * D3uu[a] - usq * D1[a] + T(3) * (KD3[a] + h0 * D1[a]));
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        A.P[p] = S2[p];
        const int a = p < 3 ? p : (p == 5 ? 1 : 0);
        const int b = p < 3 ? p : (p == 3 ? 1 : 2);
        T q = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) q += ((a == b && b == c) ? D1[a] : D3[sym3(a, b, c)]) * u[c];
        A.Qm[p] = q;
    }
    return A;
}

// v = dfeq/dj contracted with mu; G = symmetric Theta-gradient contribution (without 1/tau).
template <int Q, typename T>
__device__ __forceinline__ void adj_finish(const Coef<T>& cf, const EqCell<T>& e, const AdjAcc<T>& A, T (&v)[3],
                                           T (&G)[6]) {
    const T u[3] = {e.ux, e.uy, e.uz};
    const T c3 = cf.c3;
    const T KV[3] = {cf.K[0] * A.V[0] + cf.K[3] * A.V[1] + cf.K[4] * A.V[2],
                     cf.K[3] * A.V[0] + cf.K[1] * A.V[1] + cf.K[5] * A.V[2],
                     cf.K[4] * A.V[0] + cf.K[5] * A.V[1] + cf.K[2] * A.V[2]};
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = A.Va[a] - u[a] * A.B - T(2) * c3 * KV[a];
    const T rho = e.rho;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        G[a] = rho * (T(4.5) * (A.P[a] - A.P0 * T(1.0 / 3.0)) +
                      c3 * (T(3) * (A.Qm[a] - A.Q0 * T(1.0 / 3.0)) - T(2) * A.V[a] * u[a]));
    // off-diagonal: dL/dTheta_ab + dL/dTheta_ba
    G[3] = rho * (T(9) * A.P[3] + c3 * (T(6) * A.Qm[3] - T(2) * (A.V[0] * u[1] + A.V[1] * u[0])));
    G[4] = rho * (T(9) * A.P[4] + c3 * (T(6) * A.Qm[4] - T(2) * (A.V[0] * u[2] + A.V[2] * u[0])));
    G[5] = rho * (T(9) * A.P[5] + c3 * (T(6) * A.Qm[5] - T(2) * (A.V[1] * u[2] + A.V[2] * u[1])));
}

// Gradient record per block: [0..5] Theta (xx yy zz xy xz yz), [6] tau, [7] unused.
// Each block accumulates into its own record, in launch order, so the result is deterministic.
template <typename T>
__device__ __forceinline__ void accumulate_record(T (&v)[8], double* gpart) {
    const double s = block_sum_lane<8, T>(v);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid < 8) gpart[block_linear() * 8 + tid] += s;
}

template <int Q, int S, bool MASK, int LAYOUT>
__global__ void __launch_bounds__(256) k_adj_seed(Geom g, Coef<typename Store<S>::T> cf,
                                                  const Planes<const typename Store<S>::type> src,
                                                  const typename Store<S>::T* __restrict__ grad,
                                                  const Planes<typename Store<S>::T> lam) {
    using T = typename Store<S>::T;
    Cell c;
    if (!make_cell(g, c)) return;
    const uint32_t lw = link_of<MASK>(g, c);
    if (MASK && (lw & LINK_SOLID)) return;
    const size_t N = g.N;
    T d[Q];
    gather<Q, S, MASK, LAYOUT, true>(c, lw, cf, src, d);
    const Macro<T> m = macro_of<Q, T>(d, cf.rho0);
    const T gx = grad[c.n], gy = grad[N + c.n], gz = Lat<Q>::D == 3 ? grad[2 * N + c.n] : T(0);
    const T inv = T(1) / m.rho;
    const T gu = gx * m.ux + gy * m.uy + gz * m.uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) lam.p[i][c.n] = (vdot<T>(vel<Q>(i), gx, gy, gz) - gu) * inv;
}

// Register caps: D2Q9/D3Q19 at most 64 (four 256-thread blocks per SM instead of three; the few
// spilled values stay in L1): FP16 AA adjoint at 256^3 0.69 -> 0.77 of the copy peak, FP32 pull
// 0.87 -> 0.90 (measured). D3Q27 at most 128 (two blocks instead of one at 189 registers, no
// spills). FP64 storage is left uncapped.
template <int Q, int S, bool MASK, int LAYOUT>
__global__ void __launch_bounds__(256, S == 1 ? 1 : Q == 27 ? 2 : 4) k_adj_step(Geom g, Coef<typename Store<S>::T> cf,
                                                  const Planes<const typename Store<S>::type> src,
                                                  const Planes<const typename Store<S>::T> lam_next,
                                                  const Planes<typename Store<S>::T> lam, double* __restrict__ gpart) {
    using T = typename Store<S>::T;
    T rec[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    Cell c;
    if (make_cell(g, c)) {
        const uint32_t lw = link_of<MASK>(g, c);
        if (!(MASK && (lw & LINK_SOLID))) {
            // mu = S^T lambda_{t+1}: reverse gather along +c_i
            T mu[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T* p;
                if (i == 0)
                    p = lam_next.p[0] + c.n;
                else if (MASK && link_bit(lw, opp(i)))
                    p = lam_next.p[opp(i)] + c.n;
                else
                    p = lam_next.p[i] + off_plus(c, vel<Q>(i));
                mu[i] = __ldg(p);
            }
            // f_t: moments, and f_i itself for the tau-gradient
            T dk[Q];
            gather<Q, S, MASK, LAYOUT, true>(c, lw, cf, src, dk);
            const Macro<T> m = macro_of<Q, T>(dk, cf.rho0);
            const EqCell<T> e = eq_cell<T>(cf, m.drho, m.rho, m.ux, m.uy, m.uz);
            const AdjAcc<T> A = adj_accumulate<Q, T>(cf, e, mu, dk);
            T v[3], G[6];
            adj_finish<Q, T>(cf, e, A, v, G);
            const T om = cf.omega, om1 = T(1) - cf.omega;
            lam.p[0][c.n] = om1 * mu[0] + om * A.v0;
#pragma unroll
            for (int k = 0; k < Lat<Q>::P; ++k) {
                const int i = 2 * k + 1;
                const T cv = vdot<T>(vel<Q>(i), v[0], v[1], v[2]);
                lam.p[i][c.n] = om1 * mu[i] + om * (A.v0 + cv);
                lam.p[i + 1][c.n] = om1 * mu[i + 1] + om * (A.v0 - cv);
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) rec[k] = om * G[k];
            rec[6] = -(om * om) * A.gE;
        }
    }
    accumulate_record<T>(rec, gpart);
}

template <int Q, typename T>
__global__ void __launch_bounds__(256) k_adj_init(Geom g, Coef<T> cf, const T* __restrict__ rho0,
                                                  const T* __restrict__ u0, const Planes<const T> lam0,
                                                  T* __restrict__ du0, double* __restrict__ gpart) {
    T rec[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    Cell c;
    if (make_cell(g, c)) {
        const size_t N = g.N;
        const bool solid = g.link && (__ldg(g.link + c.n) & LINK_SOLID);
        if (solid) {
            if (du0)
                for (int a = 0; a < Lat<Q>::D; ++a) du0[a * N + c.n] = T(0);
        } else {
            const T rho = rho0 ? rho0[c.n] : cf.rho0;
            const T ux = u0 ? u0[c.n] : T(0), uy = u0 ? u0[N + c.n] : T(0);
            const T uz = (u0 && Lat<Q>::D == 3) ? u0[2 * N + c.n] : T(0);
            const EqCell<T> e = eq_cell<T>(cf, rho - cf.rho0, rho, ux, uy, uz);
            T mu[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) mu[i] = lam0.p[i][c.n];
            const AdjAcc<T> A = adj_accumulate<Q, T>(cf, e, mu, nullptr);
            T v[3], G[6];
            adj_finish<Q, T>(cf, e, A, v, G);
            if (du0)
                for (int a = 0; a < Lat<Q>::D; ++a) du0[a * N + c.n] = rho * v[a];
#pragma unroll
            for (int k = 0; k < 6; ++k) rec[k] = G[k];
        }
    }
    accumulate_record<T>(rec, gpart);
}

}  // namespace LBM_VARIANT
}  // namespace lbm
