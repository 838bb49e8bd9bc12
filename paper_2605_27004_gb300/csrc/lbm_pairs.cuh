// Two-cells-per-thread forward kernels for the FP32 and FP16 storage forms (sm_100+ packed FP32).
//
// A thread owns the x-adjacent cells (x0, x0 + 1), x0 even, of one row; a warp owns 64
// consecutive cells of one row (blocks are a multiple of 32 threads wide). Population planes
// whose velocity has c_x = 0 are read and written as aligned 2-element vectors (half2 or
// float2), which halves their load/store and address instructions per cell. Along x the pull
// gather needs f(x0 - c_x) and f(x0 + 1 - c_x), which straddle a vector boundary when
// c_x = +-1; those directions are read (and the odd AA step's scatter along +c_x is written) as
// two single elements with periodic wrap. Exchanging the straddling element with the
// neighbouring lane by a warp shuffle instead measured 1-4 % slower. The collision runs on
// (cell A, cell B) pairs with the packed FP32 instructions (FFMA2 / FADD2 / FMUL2), the same
// operation order as the one-cell kernels except that 1/tau is folded into per-cell factors
// (see bgk2).
#pragma once
#include "lbm_ade.cuh"
#include "lbm_kernels.cuh"

namespace lbm {
inline namespace LBM_VARIANT {

// ---------------------------------------------------------------------------------------------
// Packed FP32 pair arithmetic
// ---------------------------------------------------------------------------------------------
struct F2 {
    float2 v;
};
__device__ __forceinline__ F2 f2(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ F2 f2(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ F2 operator-(F2 a) { return {make_float2(-a.v.x, -a.v.y)}; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) {
    a = a + b;
    return a;
}
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) {
    a = a - b;
    return a;
}

__device__ __forceinline__ void add_c2(Vec3 v, F2 val, F2& x, F2& y, F2& z) {
    if (v.x == 1) x += val;
    if (v.x == -1) x -= val;
    if (v.y == 1) y += val;
    if (v.y == -1) y -= val;
    if (v.z == 1) z += val;
    if (v.z == -1) z -= val;
}
__device__ __forceinline__ F2 vdot2(Vec3 v, F2 ax, F2 ay, F2 az) {
    F2 r = f2(0.f);
    bool first = true;
    auto acc = [&](int s, F2 a) {
        if (s == 0) return;
        if (first) {
            r = s > 0 ? a : -a;
            first = false;
        } else if (s > 0) {
            r += a;
        } else {
            r -= a;
        }
    };
    acc(v.x, ax);
    acc(v.y, ay);
    acc(v.z, az);
    return r;
}

// ---------------------------------------------------------------------------------------------
// Storage vectors: two consecutive elements of one plane
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ F2 ld2(const float* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v};
}
__device__ __forceinline__ F2 ld2(const __half* p) {
    const unsigned int w = __ldg(reinterpret_cast<const unsigned int*>(p));
    return {__half22float2(*reinterpret_cast<const __half2*>(&w))};
}
__device__ __forceinline__ F2 ld2_rw(const float* p) { return {*reinterpret_cast<const float2*>(p)}; }
__device__ __forceinline__ F2 ld2_rw(const __half* p) {
    const unsigned int w = *reinterpret_cast<const unsigned int*>(p);
    return {__half22float2(*reinterpret_cast<const __half2*>(&w))};
}
__device__ __forceinline__ void st2(float* p, F2 v) { *reinterpret_cast<float2*>(p) = v.v; }
__device__ __forceinline__ void st2(__half* p, F2 v) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(v.v); }

template <int S>
__device__ __forceinline__ F2 to_shifted2(F2 raw, float r) {
    return Store<S>::shifted ? raw : raw - f2(r);
}
template <int S>
__device__ __forceinline__ F2 from_shifted2(F2 d, float r) {
    return Store<S>::shifted ? d : d + f2(r);
}

// Pair cell: thread (lane) owns x0 and x0 + 1 of row (y, z).
struct PCell {
    int x0, y, z;
    bool in_grid;    // the pair lies inside the grid
    bool active;     // in the grid and not entirely solid
    uint32_t n;      // index of cell x0
    uint32_t X[3];   // wrapped x0 + 1, x0, x0 - 1 (only X[1] is used for vector access)
    uint32_t R[3][3];
};

__device__ __forceinline__ void make_pcell(const Geom& g, PCell& c) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    c.x0 = 2 * px;
    c.y = blockIdx.y * blockDim.y + threadIdx.y;
    c.z = blockIdx.z + LBM_SLAB;
    c.in_grid = c.x0 < g.nx && c.y < g.ny;
    // clamp out-of-grid lanes to a valid pair so that any address they form is in bounds
    const int x0 = c.in_grid ? c.x0 : 0;
    const int y = c.y < g.ny ? c.y : 0;
    const uint32_t yy[3] = {(uint32_t)(y + 1 == g.ny ? 0 : y + 1), (uint32_t)y, (uint32_t)(y == 0 ? g.ny - 1 : y - 1)};
    const uint32_t zz[3] = {(uint32_t)(c.z + 1 == g.nz ? 0 : c.z + 1), (uint32_t)c.z,
                            (uint32_t)(c.z == 0 ? g.nz - 1 : c.z - 1)};
    const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) c.R[a][b] = nx * (yy[a] + ny * zz[b]);
    c.X[1] = (uint32_t)x0;
    c.n = (uint32_t)x0 + c.R[1][1];
    c.x0 = x0;
}

// f(x0 - cx) and f(x0 + 1 - cx) of the row at element offset `row` of plane p (pull shift).
template <int S, bool RO>
__device__ __forceinline__ F2 gather_pair(const typename Store<S>::type* p, uint32_t row, const PCell& c, int cx,
                                          int nx, float r) {
    F2 v = f2(0.f);
    if (c.active) {
        if (cx == 0) {
            v = RO ? ld2(p + row + c.x0) : ld2_rw(p + row + c.x0);
        } else {
            const int xa = cx == 1 ? (c.x0 == 0 ? nx - 1 : c.x0 - 1) : c.x0 + 1;
            const int xb = cx == 1 ? c.x0 : (c.x0 + 2 == nx ? 0 : c.x0 + 2);
            v = f2(RO ? ld_ro(p + row + xa) : ld_rw(p + row + xa), RO ? ld_ro(p + row + xb) : ld_rw(p + row + xb));
        }
    }
    return to_shifted2<S>(v, r);
}

// ---------------------------------------------------------------------------------------------
// Pair collision: the arithmetic of bgk<Q, float, FIX> on two cells per instruction, with 1/tau
// folded into the per-cell factors (om drho, om rho, om 4.5 rho) and 2 K~.u precomputed, so that
// the relaxed value of each population is one FFMA2 away from its pair's even/odd parts. Rounding
// differs from the one-cell kernels in the last bits; the shorter per-pair dependency chains are
// worth 0.745 -> 0.82 of the copy peak at 256^3 for FP16 storage (measured).
// ---------------------------------------------------------------------------------------------
struct Macro2 {
    F2 drho, rho, jx, jy, jz, ux, uy, uz;
};

// Relaxation of a pair towards feq(rho, u) in shifted variables (drho = rho - rho0), with 1/tau
// folded into the per-cell factors and 2 K~.u precomputed (see the file comment).
template <int Q>
__device__ __forceinline__ void relax2(const Coef<float>& cf, F2 drho, F2 rho, F2 ux, F2 uy, F2 uz, F2 (&d)[Q]) {
    const F2 usq = fma2(ux, ux, fma2(uy, uy, uz * uz));
    const F2 kx = fma2(f2(cf.K[0]), ux, fma2(f2(cf.K[3]), uy, f2(cf.K[4]) * uz));
    const F2 ky = fma2(f2(cf.K[3]), ux, fma2(f2(cf.K[1]), uy, f2(cf.K[5]) * uz));
    const F2 kz = fma2(f2(cf.K[4]), ux, fma2(f2(cf.K[5]), uy, f2(cf.K[2]) * uz));
    const F2 r45 = f2(4.5f) * rho;
    const F2 usq3 = usq * f2(1.0f / 3.0f);
    const F2 om = f2(cf.omega), om1 = f2(1.f - cf.omega);
    const F2 omdrho = om * drho, omrho = om * rho, omr45 = om * r45;
    const F2 kx2 = f2(2.f) * kx, ky2 = f2(2.f) * ky, kz2 = f2(2.f) * kz;
    {
        const F2 feq = fma2(omdrho, f2(cf.A[0]), -(f2((float)weight<Q>(0)) * omr45 * usq3));
        d[0] = fma2(om1, d[0], feq);
    }
#pragma unroll
    for (int k = 0; k < Lat<Q>::P; ++k) {
        const int i = 2 * k + 1;
        const Vec3 v = vel<Q>(i);
        const F2 w = f2((float)weight<Q>(i));
        const F2 uc = vdot2(v, ux, uy, uz);
        const F2 qk2 = vdot2(v, kx2, ky2, kz2);
        const F2 E = fma2(omdrho, f2(cf.A[i]), (w * omr45) * fma2(uc, uc, -usq3));
        const F2 cub = fma2(uc, fma2(uc, uc, -usq), -qk2);
        const F2 O = omrho * fma2(uc, f2(cf.B[i]), f2(cf.c3 * (float)weight<Q>(i)) * cub);
        d[i] = fma2(om1, d[i], E + O);
        d[i + 1] = fma2(om1, d[i + 1], E - O);
    }
}

template <int Q, bool FIX>
__device__ __forceinline__ Macro2 bgk2(const Coef<float>& cf, F2 (&d)[Q]) {
    Macro2 m;
    F2 s = d[0], jx = f2(0.f), jy = f2(0.f), jz = f2(0.f);
#pragma unroll
    for (int k = 0; k < Lat<Q>::P; ++k) {
        const F2 a = d[2 * k + 1], b = d[2 * k + 2];
        s += a + b;
        add_c2(vel<Q>(2 * k + 1), a - b, jx, jy, jz);
    }
    m.drho = s;
    m.rho = f2(cf.rho0) + s;
    m.jx = jx;
    m.jy = jy;
    m.jz = jz;
    const F2 inv = f2(1.f / m.rho.v.x, 1.f / m.rho.v.y);
    m.ux = jx * inv;
    m.uy = jy * inv;
    m.uz = Lat<Q>::D == 3 ? jz * inv : f2(0.f);
    relax2<Q>(cf, m.drho, m.rho, m.ux, m.uy, m.uz, d);
    if (FIX) {
        F2 ex = -m.jx, ey = -m.jy, ez = -m.jz;
#pragma unroll
        for (int k = 0; k < Lat<Q>::P; ++k) add_c2(vel<Q>(2 * k + 1), d[2 * k + 1] - d[2 * k + 2], ex, ey, ez);
#pragma unroll
        for (int k = 0; k < Lat<Q>::P; ++k) {
            const Vec3 v = vel<Q>(2 * k + 1);
            const F2 corr = f2((float)(3.0 * weight<Q>(2 * k + 1))) * vdot2(v, ex, ey, ez);
            d[2 * k + 1] -= corr;
            d[2 * k + 2] += corr;
        }
    }
    return m;
}

__device__ __forceinline__ bool bad1(float rho, float ux, float uy, float uz) {
    return !(rho > 0.f) || !isfinite(ux + uy + uz);
}

// Collision of the pair at cell index n (even): the flow's BGK, or (ADE) the advection-diffusion
// relaxation of a scalar with the prescribed velocity read as one aligned vector per component
// (lbm_ade.cuh). Returns true when a fluid cell of the pair (fa, fb) is unstable.
template <int Q, int S, bool ADE>
__device__ __forceinline__ bool collide2(const Coef<float>& cf, const VelField<float>& vf, uint32_t n, F2 (&d)[Q],
                                         bool fa, bool fb) {
    if constexpr (ADE) {
        F2 ux = f2(0.f), uy = f2(0.f), uz = f2(0.f);
        if (vf.p[0] != nullptr) {
            ux = ld2(vf.p[0] + n);
            uy = ld2(vf.p[1] + n);
            if (Lat<Q>::D == 3) uz = ld2(vf.p[2] + n);
        }
        F2 s = d[0];
#pragma unroll
        for (int k = 0; k < Lat<Q>::P; ++k) s += d[2 * k + 1] + d[2 * k + 2];
        relax2<Q>(cf, s, f2(cf.rho0) + s, ux, uy, uz, d);
        return (fa && !isfinite(s.v.x)) || (fb && !isfinite(s.v.y));
    } else {
        const Macro2 m = bgk2<Q, Store<S>::fix_momentum>(cf, d);
        return (fa && bad1(m.rho.v.x, m.ux.v.x, m.uy.v.x, m.uz.v.x)) ||
               (fb && bad1(m.rho.v.y, m.ux.v.y, m.uy.v.y, m.uz.v.y));
    }
}

// ---------------------------------------------------------------------------------------------
// Pull step, two cells per thread. The D3Q27 pair kernels run blocks of 128 threads, five per SM
// at 96 registers (8-48 bytes of spills): 20 resident warps instead of 16 with two 256-thread
// blocks at 126 registers, measured at 256^3 / 384^3 pull 0.774 -> 0.828 / 0.780 -> 0.827 of the
// copy peak, AA 0.715 -> 0.788 / 0.728 -> 0.787 (which also moved the odd AA step from one cell
// per thread to pairs).
// ---------------------------------------------------------------------------------------------
template <int Q>
constexpr int pair_threads() {
    return Q == 27 ? 128 : 256;
}

template <int Q, int S, bool MASK, bool ADE = false>
__global__ void __launch_bounds__(pair_threads<Q>(), Q == 27 ? 5 : (S != 3 ? 2 : 3))
    k_step_pull2(Geom g, Coef<float> cf, VelField<float> vf, const Planes<const typename Store<S>::type> src,
                 const Planes<typename Store<S>::type> dst, int* __restrict__ flag) {
    PCell c;
    make_pcell(g, c);
    uint2 lw = make_uint2(0u, 0u);
    if (MASK && c.in_grid) lw = __ldg(reinterpret_cast<const uint2*>(g.link + c.n));
    const bool fa = !(lw.x & LINK_SOLID), fb = !(lw.y & LINK_SOLID);
    c.active = c.in_grid && (fa || fb);
    F2 d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const Vec3 v = vel<Q>(i);
        d[i] = gather_pair<S, true>(src.p[i], c.R[v.y + 1][v.z + 1], c, v.x, g.nx, cf.so[i]);
        if (MASK && i > 0) {
            const bool wa = link_bit(lw.x, i), wb = link_bit(lw.y, i);
            if (c.active && (wa || wb)) {  // half-way bounce-back from the own cell's opposite slot
                const F2 own = to_shifted2<S>(ld2(src.p[opp(i)] + c.n), cf.so[i]);
                d[i] = f2(wa ? own.v.x : d[i].v.x, wb ? own.v.y : d[i].v.y);
            }
        }
    }
    if (!c.active) return;
    if (collide2<Q, S, ADE>(cf, vf, c.n, d, fa, fb)) *flag = 1;
    if (!MASK || (fa && fb)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) st2(dst.p[i] + c.n, from_shifted2<S>(d[i], cf.so[i]));
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const F2 o = from_shifted2<S>(d[i], cf.so[i]);
            if (fa) st_raw(dst.p[i] + c.n, o.v.x);
            if (fb) st_raw(dst.p[i] + c.n + 1, o.v.y);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// AA even step (state LOCAL -> AAODD), two cells per thread: purely local.
// ---------------------------------------------------------------------------------------------
template <int Q, int S, bool MASK, bool ADE = false>
__global__ void __launch_bounds__(pair_threads<Q>(), Q == 27 ? 5 : (S != 3 ? 2 : 3))
    k_step_aa_even2(Geom g, Coef<float> cf, VelField<float> vf, const Planes<const typename Store<S>::type> src,
                    const Planes<typename Store<S>::type> dst, int* __restrict__ flag) {
    PCell c;
    make_pcell(g, c);
    if (!c.in_grid) return;
    uint2 lw = make_uint2(0u, 0u);
    if (MASK) lw = __ldg(reinterpret_cast<const uint2*>(g.link + c.n));
    const bool fa = !(lw.x & LINK_SOLID), fb = !(lw.y & LINK_SOLID);
    if (!fa && !fb) return;
    F2 d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = to_shifted2<S>(ld2_rw(src.p[i] + c.n), cf.so[i]);
    if (collide2<Q, S, ADE>(cf, vf, c.n, d, fa, fb)) *flag = 1;
    if (!MASK || (fa && fb)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) st2(dst.p[opp(i)] + c.n, from_shifted2<S>(d[i], cf.so[i]));
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const F2 o = from_shifted2<S>(d[i], cf.so[i]);
            if (fa) st_raw(dst.p[opp(i)] + c.n, o.v.x);
            if (fb) st_raw(dst.p[opp(i)] + c.n + 1, o.v.y);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// AA odd step (state AAODD -> LOCAL), two cells per thread, boxes without walls. Gather
// f_i(x) = A[opp i][x - c_i] as in the pull step; scatter f*_i(x) to A[i][x + c_i]. Along x the
// targets of (x0, x0 + 1) are shifted by c_x, so those directions are stored as two single
// elements (x0 + c_x, x0 + 1 + c_x), with periodic wrap; the others as one aligned vector.
// The old value of slot (i, x + c_i) is the population f_opp(i)(x) of the same cell, gathered by
// this thread; the store depends on that value through the collision, so every slot is read
// before it is replaced, by the only thread that writes it: in place and race free. (A thread's
// vector loads may also fetch an element that another thread consumes and replaces; such an
// element is never used by the fetching thread.)
// ---------------------------------------------------------------------------------------------
template <int Q, int S, bool ADE = false>
__global__ void __launch_bounds__(pair_threads<Q>(), Q == 27 ? 5 : (S != 3 ? 2 : 3))
    k_step_aa_odd2(Geom g, Coef<float> cf, VelField<float> vf, const Planes<const typename Store<S>::type> src,
                   const Planes<typename Store<S>::type> dst, int* __restrict__ flag) {
    PCell c;
    make_pcell(g, c);
    c.active = c.in_grid;
    F2 d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const Vec3 v = vel<Q>(i);
        d[i] = gather_pair<S, false>(src.p[opp(i)], c.R[v.y + 1][v.z + 1], c, v.x, g.nx, cf.so[i]);
    }
    if (c.active && collide2<Q, S, ADE>(cf, vf, c.n, d, true, true)) *flag = 1;
    const int nx = g.nx;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const Vec3 v = vel<Q>(i);
        const F2 o = from_shifted2<S>(d[i], cf.so[i]);
        typename Store<S>::type* row = dst.p[i] + c.R[1 - v.y][1 - v.z];  // row of x + c_i
        if (v.x == 0) {
            if (c.active) st2(row + c.x0, o);
        } else if (v.x == 1) {  // targets x0 + 1 (A) and x0 + 2 (B)
            if (c.active) {
                st_raw(row + c.x0 + 1, o.v.x);
                st_raw(row + (c.x0 + 2 == nx ? 0 : c.x0 + 2), o.v.y);
            }
        } else {  // targets x0 - 1 (A) and x0 (B)
            if (c.active) {
                st_raw(row + (c.x0 == 0 ? nx - 1 : c.x0 - 1), o.v.x);
                st_raw(row + c.x0, o.v.y);
            }
        }
    }
}

inline Shape shape_pairs(const Geom& g, int threads = 256) {
    Shape s;
    const int np = g.nx / 2;
    const int bx = block_x_for(np, threads);
    const int by = std::max(1, threads / bx);
    s.block = dim3(bx, by, 1);
    s.grid = dim3((np + bx - 1) / bx, (g.ny + by - 1) / by, g.nz - 2 * LBM_SLAB);
    s.nblocks = (long long)s.grid.x * s.grid.y * s.grid.z;
    return s;
}

}  // namespace LBM_VARIANT
}  // namespace lbm
