// Four-cells-per-thread forward kernels for FP16 storage without walls (D2Q9, D3Q19; nx a
// multiple of 4).
//
// A thread owns the cells x0 .. x0 + 3 (x0 a multiple of 4) of one row, a warp 128 consecutive
// cells. Every population plane is read as aligned 8-byte words of four halves: for c_x = 0 the
// thread's own word; for c_x = +-1 the own word and the neighbouring word on the side the shift
// comes from, from which the shifted window of four halves is cut with two byte permutations (the
// neighbouring word is the adjacent lane's, so the second load hits L1). Stores of the pull and
// the even AA step are one aligned 8-byte word per plane; the odd AA step scatters along +c_i and
// completes each thread's aligned word of an x-shifted plane with one value from the neighbouring
// lane (warp shuffle). Per cell this halves
// the load, store, address and conversion instructions of the two-cells-per-thread kernels, which
// are instruction-bound for FP16 storage. The collision is the packed pair collision (collide2:
// the flow's BGK, or with ADE the scalar's relaxation with the prescribed velocity read as aligned
// float2 pairs) on (x0, x0 + 1) and then on (x0 + 2, x0 + 3).
#pragma once
#include "lbm_pairs.cuh"

namespace lbm {
inline namespace LBM_VARIANT {

struct QCell {
    int x0, y, z;
    bool active;  // the four cells lie inside the grid
    uint32_t n;   // index of cell x0
    uint32_t R[3][3];
};

__device__ __forceinline__ void make_qcell(const Geom& g, QCell& c) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    c.x0 = 4 * px;
    c.y = blockIdx.y * blockDim.y + threadIdx.y;
    c.z = blockIdx.z + LBM_SLAB;
    c.active = c.x0 < g.nx && c.y < g.ny;
    const int x0 = c.active ? c.x0 : 0;  // inactive lanes address a valid word and load nothing
    const int y = c.y < g.ny ? c.y : 0;
    const uint32_t yy[3] = {(uint32_t)(y + 1 == g.ny ? 0 : y + 1), (uint32_t)y, (uint32_t)(y == 0 ? g.ny - 1 : y - 1)};
    const uint32_t zz[3] = {(uint32_t)(c.z + 1 == g.nz ? 0 : c.z + 1), (uint32_t)c.z,
                            (uint32_t)(c.z == 0 ? g.nz - 1 : c.z - 1)};
    const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) c.R[a][b] = nx * (yy[a] + ny * zz[b]);
    c.n = (uint32_t)x0 + c.R[1][1];
    c.x0 = x0;
}

template <bool RO>
__device__ __forceinline__ uint2 ld_word4(const __half* p) {
    return RO ? __ldg(reinterpret_cast<const uint2*>(p)) : *reinterpret_cast<const uint2*>(p);
}
__device__ __forceinline__ F2 half2_bits_to_f2(unsigned w) {
    __half2 h;
    memcpy(&h, &w, sizeof(w));
    return {__half22float2(h)};
}
__device__ __forceinline__ unsigned f2_to_half2_bits(F2 v) {
    const __half2 h = __float22half2_rn(v.v);
    unsigned w;
    memcpy(&w, &h, sizeof(w));
    return w;
}
// halves (hi of a, lo of b): the window one half to the right of the word pair (a, b)
__device__ __forceinline__ unsigned mid_halves(unsigned a, unsigned b) { return __byte_perm(a, b, 0x5432); }

// f(x0 - cx) .. f(x0 + 3 - cx) of the row at element offset `row` of plane p, as the pairs
// (cells x0, x0 + 1) -> a and (x0 + 2, x0 + 3) -> b.
template <bool RO>
__device__ __forceinline__ void gather_quad(const __half* p, uint32_t row, const QCell& c, int cx, int nx, F2& a,
                                            F2& b) {
    if (!c.active) {
        a = b = f2(0.f);
        return;
    }
    const __half* r = p + row;
    const uint2 cur = ld_word4<RO>(r + c.x0);
    if (cx == 0) {
        a = half2_bits_to_f2(cur.x);
        b = half2_bits_to_f2(cur.y);
    } else if (cx == 1) {  // x0 - 1 .. x0 + 2
        const uint2 prev = ld_word4<RO>(r + (c.x0 == 0 ? nx - 4 : c.x0 - 4));
        a = half2_bits_to_f2(mid_halves(prev.y, cur.x));
        b = half2_bits_to_f2(mid_halves(cur.x, cur.y));
    } else {  // x0 + 1 .. x0 + 4
        const uint2 next = ld_word4<RO>(r + (c.x0 + 4 == nx ? 0 : c.x0 + 4));
        a = half2_bits_to_f2(mid_halves(cur.x, cur.y));
        b = half2_bits_to_f2(mid_halves(cur.y, next.x));
    }
}

__device__ __forceinline__ void st_word4(__half* p, F2 a, F2 b) {
    *reinterpret_cast<uint2*>(p) = make_uint2(f2_to_half2_bits(a), f2_to_half2_bits(b));
}

// ---------------------------------------------------------------------------------------------
// Pull step, four cells per thread (FP16 r-shifted storage: the stored value is d = f - r).
// ---------------------------------------------------------------------------------------------
template <int Q, bool ADE = false>
__global__ void __launch_bounds__(256, 2)
    k_step_pull4(Geom g, Coef<float> cf, VelField<float> vf, const Planes<const __half> src, const Planes<__half> dst,
                 int* __restrict__ flag) {
    QCell c;
    make_qcell(g, c);
    F2 da[Q], db[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const Vec3 v = vel<Q>(i);
        gather_quad<true>(src.p[i], c.R[v.y + 1][v.z + 1], c, v.x, g.nx, da[i], db[i]);
    }
    if (!c.active) return;
    const bool bad = collide2<Q, 3, ADE>(cf, vf, c.n, da, true, true) | collide2<Q, 3, ADE>(cf, vf, c.n + 2, db, true, true);
    if (bad) *flag = 1;
#pragma unroll
    for (int i = 0; i < Q; ++i) st_word4(dst.p[i] + c.n, da[i], db[i]);
}

// ---------------------------------------------------------------------------------------------
// AA even step (state LOCAL -> AAODD), four cells per thread: purely local, aligned words.
// ---------------------------------------------------------------------------------------------
template <int Q, bool ADE = false>
__global__ void __launch_bounds__(256, 2)
    k_step_aa_even4(Geom g, Coef<float> cf, VelField<float> vf, const Planes<const __half> src, const Planes<__half> dst,
                    int* __restrict__ flag) {
    QCell c;
    make_qcell(g, c);
    if (!c.active) return;
    F2 da[Q], db[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint2 w = ld_word4<false>(src.p[i] + c.n);
        da[i] = half2_bits_to_f2(w.x);
        db[i] = half2_bits_to_f2(w.y);
    }
    const bool bad = collide2<Q, 3, ADE>(cf, vf, c.n, da, true, true) | collide2<Q, 3, ADE>(cf, vf, c.n + 2, db, true, true);
    if (bad) *flag = 1;
#pragma unroll
    for (int i = 0; i < Q; ++i) st_word4(dst.p[opp(i)] + c.n, da[i], db[i]);
}

// ---------------------------------------------------------------------------------------------
// AA odd step (state AAODD -> LOCAL), four cells per thread: gather f_i(x) = A[opp i][x - c_i]
// as in the pull step, scatter f*_i(x) to A[i][x + c_i]. For c_x = +-1 the four targets
// x0 + c_x .. x0 + 3 + c_x straddle a word boundary: one half, one aligned 4-byte word of two
// halves, one half (with periodic wrap). Each slot this thread writes holds a population this
// thread gathered (the one of the opposite direction at the same cell), so the update is in
// place and race free; elements of the neighbouring words that a thread loads but does not own
// are never used by it.
// ---------------------------------------------------------------------------------------------
template <int Q, bool ADE = false>
__global__ void __launch_bounds__(256, 2)
    k_step_aa_odd4(Geom g, Coef<float> cf, VelField<float> vf, const Planes<const __half> src, const Planes<__half> dst,
                   int* __restrict__ flag) {
    QCell c;
    make_qcell(g, c);
    F2 da[Q], db[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const Vec3 v = vel<Q>(i);
        gather_quad<false>(src.p[opp(i)], c.R[v.y + 1][v.z + 1], c, v.x, g.nx, da[i], db[i]);
    }
    if (!c.active) return;
    const bool bad = collide2<Q, 3, ADE>(cf, vf, c.n, da, true, true) | collide2<Q, 3, ADE>(cf, vf, c.n + 2, db, true, true);
    if (bad) *flag = 1;
    const int nx = g.nx;
    // Rows are multiples of 128 cells (quads()), so a warp is 32 threads of one row, its lane 0 the
    // row start or the successor of another warp's lane 31. For c_x = +-1 the value that belongs to
    // the thread's own aligned word but comes from the neighbouring lane's cell is taken by a warp
    // shuffle, and the word is stored whole; only the warp's end lanes store single halves across
    // the warp boundary. Each slot is still written after the lane that gathered it has gathered it:
    // the shuffled value depends on that lane's gather (measured for the flow at 256^3 / 512^3 /
    // 768^3: AA 0.843 -> 0.854 / 0.864 -> 0.888 / 0.874 -> 0.867).
    const int lane = (threadIdx.x + threadIdx.y * blockDim.x) & 31;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const Vec3 v = vel<Q>(i);
        __half* row = dst.p[i] + c.R[1 - v.y][1 - v.z];  // row of x + c_i
        if (v.x == 0) {
            st_word4(row + c.x0, da[i], db[i]);
            continue;
        }
        const unsigned wa = f2_to_half2_bits(da[i]), wb = f2_to_half2_bits(db[i]);
        if constexpr (ADE) {  // the scalar keeps the three stores per plane (measured 0.851 -> 0.833 with shuffles)
            const int xf = v.x == 1 ? c.x0 + 1 : (c.x0 == 0 ? nx - 1 : c.x0 - 1);
            const int xm = v.x == 1 ? c.x0 + 2 : c.x0;
            const int xl = v.x == 1 ? (c.x0 + 4 == nx ? 0 : c.x0 + 4) : c.x0 + 2;
            *reinterpret_cast<unsigned short*>(row + xf) = (unsigned short)(wa & 0xffffu);
            *reinterpret_cast<unsigned*>(row + xm) = mid_halves(wa, wb);
            *reinterpret_cast<unsigned short*>(row + xl) = (unsigned short)(wb >> 16);
        } else if (v.x == 1) {  // targets x0 + 1 .. x0 + 4: own word gets (lane - 1's last, a.x, a.y, b.x)
            const unsigned prev = __shfl_up_sync(0xffffffffu, wb >> 16, 1);
            if (lane != 0) {
                *reinterpret_cast<uint2*>(row + c.x0) = make_uint2((prev & 0xffffu) | (wa << 16), mid_halves(wa, wb));
            } else {
                *reinterpret_cast<unsigned short*>(row + c.x0 + 1) = (unsigned short)(wa & 0xffffu);
                *reinterpret_cast<unsigned*>(row + c.x0 + 2) = mid_halves(wa, wb);
            }
            if (lane == 31)  // into the next warp's word (or the row start)
                *reinterpret_cast<unsigned short*>(row + (c.x0 + 4 == nx ? 0 : c.x0 + 4)) = (unsigned short)(wb >> 16);
        } else {  // targets x0 - 1 .. x0 + 2: own word gets (a.y, b.x, b.y, lane + 1's first)
            const unsigned next = __shfl_down_sync(0xffffffffu, wa & 0xffffu, 1);
            if (lane != 31) {
                *reinterpret_cast<uint2*>(row + c.x0) = make_uint2(mid_halves(wa, wb), (wb >> 16) | (next << 16));
            } else {
                *reinterpret_cast<unsigned*>(row + c.x0) = mid_halves(wa, wb);
                *reinterpret_cast<unsigned short*>(row + c.x0 + 2) = (unsigned short)(wb >> 16);
            }
            if (lane == 0)  // into the previous warp's word (or the row end)
                *reinterpret_cast<unsigned short*>(row + (c.x0 == 0 ? nx - 1 : c.x0 - 1)) = (unsigned short)(wa & 0xffffu);
        }
    }
}

inline Shape shape_quads(const Geom& g) {
    Shape s;
    const int nq = g.nx / 4;
    const int bx = block_x_for(nq);
    const int by = std::max(1, 256 / bx);
    s.block = dim3(bx, by, 1);
    s.grid = dim3((nq + bx - 1) / bx, (g.ny + by - 1) / by, g.nz - 2 * LBM_SLAB);
    s.nblocks = (long long)s.grid.x * s.grid.y * s.grid.z;
    return s;
}

}  // namespace LBM_VARIANT
}  // namespace lbm
