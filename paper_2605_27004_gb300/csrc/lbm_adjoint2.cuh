// Two-cells-per-thread adjoint step for FP16-shifted storage without walls (sm_100+ packed FP32).
//
// The same step as k_adj_step (reverse gather of lambda_(t+1), transposed Jacobian of the
// anisotropic BGK collision through the moments of mu, Theta/tau gradient records), with each
// thread owning the x-adjacent cells (x0, x0 + 1): c_x = 0 planes of lambda and of f_t are read
// and lambda_t is written as aligned 2-element vectors, x-shifted planes as two single elements
// with periodic wrap, and the arithmetic runs on (cell A, cell B) pairs with the packed FP32
// instructions. The two lanes of each gradient record are added in FP32 before the block sum.
// Blocks of 128 threads, five per SM at 96 registers (about 120 bytes of spills): 20 resident
// warps instead of 16 with two 256-thread blocks at 126 registers, measured for the FP16 AA
// adjoint at 256^3 / 512^3: 0.818 -> 0.875 / 0.831 -> 0.885 of the copy peak (266 B per cell).
#pragma once
#include "lbm_pairs.cuh"

namespace lbm {
inline namespace LBM_VARIANT {

// lambda_(t+1),i at x0 + c_i and x0 + 1 + c_i (reverse gather), row of x + c_i at `row`
__device__ __forceinline__ F2 gather_lam(const float* p, uint32_t row, const PCell& c, int cx, int nx) {
    if (cx == 0) return ld2(p + row + c.x0);
    const int xa = cx == 1 ? c.x0 + 1 : (c.x0 == 0 ? nx - 1 : c.x0 - 1);
    const int xb = cx == 1 ? (c.x0 + 2 == nx ? 0 : c.x0 + 2) : c.x0;
    return f2(__ldg(p + row + xa), __ldg(p + row + xb));
}

template <int Q, int S, int LAYOUT>
__global__ void __launch_bounds__(128, 5)
    k_adj_step2(Geom g, Coef<float> cf, const Planes<const typename Store<S>::type> src,
                const Planes<const float> lam_next, const Planes<float> lam, double* __restrict__ gpart) {
    constexpr int D = Lat<Q>::D;
    PCell c;
    make_pcell(g, c);
    c.active = c.in_grid;
    float rec[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (c.in_grid) {
        F2 mu[Q], dk[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Vec3 v = vel<Q>(i);
            mu[i] = gather_lam(lam_next.p[i], c.R[1 - v.y][1 - v.z], c, v.x, g.nx);
            if (LAYOUT == LAYOUT_LOCAL)
                dk[i] = to_shifted2<S>(ld2(src.p[i] + c.n), cf.so[i]);
            else if (LAYOUT == LAYOUT_PULL)
                dk[i] = gather_pair<S, true>(src.p[i], c.R[v.y + 1][v.z + 1], c, v.x, g.nx, cf.so[i]);
            else
                dk[i] = gather_pair<S, true>(src.p[opp(i)], c.R[v.y + 1][v.z + 1], c, v.x, g.nx, cf.so[i]);
        }
        // moments of f_t
        F2 drho = dk[0], jx = f2(0.f), jy = f2(0.f), jz = f2(0.f);
#pragma unroll
        for (int k = 0; k < Lat<Q>::P; ++k) {
            drho += dk[2 * k + 1] + dk[2 * k + 2];
            add_c2(vel<Q>(2 * k + 1), dk[2 * k + 1] - dk[2 * k + 2], jx, jy, jz);
        }
        const F2 rho = f2(cf.rho0) + drho;
        const F2 inv = f2(1.f / rho.v.x, 1.f / rho.v.y);
        const F2 u[3] = {jx * inv, jy * inv, D == 3 ? jz * inv : f2(0.f)};
        const F2 usq = fma2(u[0], u[0], fma2(u[1], u[1], u[2] * u[2]));
        const F2 kx = fma2(f2(cf.K[0]), u[0], fma2(f2(cf.K[3]), u[1], f2(cf.K[4]) * u[2]));
        const F2 ky = fma2(f2(cf.K[3]), u[0], fma2(f2(cf.K[1]), u[1], f2(cf.K[5]) * u[2]));
        const F2 kz = fma2(f2(cf.K[4]), u[0], fma2(f2(cf.K[5]), u[1], f2(cf.K[2]) * u[2]));
        const F2 r45 = f2(4.5f) * rho;
        const F2 usq3 = usq * f2(1.0f / 3.0f);
        // moments of mu and the per-direction tau-gradient differences (see adj_accumulate)
        const F2 w0 = f2((float)weight<Q>(0));
        F2 S0 = w0 * mu[0];
        F2 gE = mu[0] * (fma2(drho, f2(cf.A[0]), -(w0 * r45 * usq3)) - dk[0]);
        F2 S2[6], D1[3], D3[7];
#pragma unroll
        for (int k = 0; k < 6; ++k) S2[k] = f2(0.f);
#pragma unroll
        for (int a = 0; a < 3; ++a) D1[a] = f2(0.f);
#pragma unroll
        for (int k = 0; k < 7; ++k) D3[k] = f2(0.f);
#pragma unroll
        for (int k = 0; k < Lat<Q>::P; ++k) {
            const int i = 2 * k + 1;
            const Vec3 v = vel<Q>(i);
            const int cc[3] = {v.x, v.y, v.z};
            const F2 w = f2((float)weight<Q>(i));
            const F2 uc = vdot2(v, u[0], u[1], u[2]);
            const F2 qk = vdot2(v, kx, ky, kz);
            const F2 E = fma2(drho, f2(cf.A[i]), (w * r45) * fma2(uc, uc, -usq3));
            const F2 cub = fma2(uc, fma2(uc, uc, -usq), -(f2(2.f) * qk));
            const F2 O = rho * fma2(uc, f2(cf.B[i]), f2(cf.c3 * (float)weight<Q>(i)) * cub);
            gE = fma2(mu[i], (E + O) - dk[i], fma2(mu[i + 1], (E - O) - dk[i + 1], gE));
            const F2 sm = w * (mu[i] + mu[i + 1]), dm = w * (mu[i] - mu[i + 1]);
            S0 += sm;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (cc[a] == 1) D1[a] += dm;
                if (cc[a] == -1) D1[a] -= dm;
#pragma unroll
                for (int b = a; b < 3; ++b) {
                    const int p2 = cc[a] * cc[b];
                    if (p2 == 1) S2[sym2(a, b)] += sm;
                    if (p2 == -1) S2[sym2(a, b)] -= sm;
#pragma unroll
                    for (int e = b; e < 3; ++e) {
                        if (a == b && b == e) continue;
                        const int p3 = cc[a] * cc[b] * cc[e];
                        if (p3 == 1) D3[sym3(a, b, e)] += dm;
                        if (p3 == -1) D3[sym3(a, b, e)] -= dm;
                    }
                }
            }
        }
        // contractions with u and K~ (see adj_accumulate) and the finish (adj_finish)
        const F2 c3 = f2(cf.c3), h0 = f2(cf.h[0]);
        F2 Q0 = f2(0.f);
#pragma unroll
        for (int a = 0; a < D; ++a) Q0 = fma2(u[a], D1[a], Q0);
        const F2 B = fma2(f2(3.f), S0, f2(2.f) * c3 * Q0);
        F2 S2u[3], D3uu[3], KD3[3];
        F2 uS2u = f2(0.f), KS2 = f2(0.f), D3uuu = f2(0.f);
#pragma unroll
        for (int a = 0; a < 3; ++a) S2u[a] = D3uu[a] = KD3[a] = f2(0.f);
#pragma unroll
        for (int a = 0; a < D; ++a) {
#pragma unroll
            for (int b = 0; b < D; ++b) {
                S2u[a] = fma2(S2[sym2(a, b)], u[b], S2u[a]);
                KS2 = fma2(f2(cf.K[sym2(a, b)]), S2[sym2(a, b)], KS2);
#pragma unroll
                for (int e = 0; e < D; ++e) {
                    const F2 t = (a == b && b == e) ? D1[a] : D3[sym3(a, b, e)];
                    D3uu[a] = fma2(t, u[b] * u[e], D3uu[a]);
                    KD3[a] = fma2(f2(cf.K[sym2(b, e)]), t, KD3[a]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            uS2u = fma2(u[a], S2u[a], uS2u);
            D3uuu = fma2(u[a], D3uu[a], D3uuu);
        }
        const F2 v0 = fma2(f2(1.f) + f2(1.5f) * usq, S0,
                           f2(4.5f) * (KS2 + h0 * S0) - f2(4.5f) * uS2u - f2(2.f) * c3 * (D3uuu - usq * Q0));
        F2 Va[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            Va[a] = f2(3.f) * D1[a] + f2(9.f) * S2u[a] +
                    c3 * (f2(3.f) * D3uu[a] - usq * D1[a] + f2(3.f) * (KD3[a] + h0 * D1[a]));
        const F2 KV[3] = {fma2(f2(cf.K[0]), D1[0], fma2(f2(cf.K[3]), D1[1], f2(cf.K[4]) * D1[2])),
                          fma2(f2(cf.K[3]), D1[0], fma2(f2(cf.K[1]), D1[1], f2(cf.K[5]) * D1[2])),
                          fma2(f2(cf.K[4]), D1[0], fma2(f2(cf.K[5]), D1[1], f2(cf.K[2]) * D1[2]))};
        F2 vv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) vv[a] = Va[a] - u[a] * B - f2(2.f) * c3 * KV[a];
        // lambda_t = (1 - 1/tau) mu + (1/tau) (v0 + c.v)
        const F2 om = f2(cf.omega), om1 = f2(1.f - cf.omega);
        st2(lam.p[0] + c.n, fma2(om1, mu[0], om * v0));
#pragma unroll
        for (int k = 0; k < Lat<Q>::P; ++k) {
            const int i = 2 * k + 1;
            const F2 cv = vdot2(vel<Q>(i), vv[0], vv[1], vv[2]);
            st2(lam.p[i] + c.n, fma2(om1, mu[i], om * (v0 + cv)));
            st2(lam.p[i + 1] + c.n, fma2(om1, mu[i + 1], om * (v0 - cv)));
        }
        // gradient records (adj_finish): Theta (xx yy zz xy xz yz) and tau
        const F2 third = f2(1.0f / 3.0f);
        F2 G[6];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            F2 Qma = f2(0.f);
            if (a < D) {
#pragma unroll
                for (int e = 0; e < D; ++e) Qma = fma2((a == e) ? D1[a] : D3[sym3(a, a, e)], u[e], Qma);
            }
            G[a] = rho * (f2(4.5f) * (S2[a] - S0 * third) + c3 * (f2(3.f) * (Qma - Q0 * third) - f2(2.f) * D1[a] * u[a]));
        }
        const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const int a = pa[p], b = pb[p];
            F2 q = f2(0.f);
#pragma unroll
            for (int e = 0; e < D; ++e) q = fma2((a == b && b == e) ? D1[a] : D3[sym3(a, b, e)], u[e], q);
            G[3 + p] = rho * (f2(9.f) * S2[3 + p] + c3 * (f2(6.f) * q - f2(2.f) * (D1[a] * u[b] + D1[b] * u[a])));
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const F2 r = om * G[k];
            rec[k] = r.v.x + r.v.y;
        }
        const F2 rt = -(om * om) * gE;
        rec[6] = rt.v.x + rt.v.y;
    }
    accumulate_record<float>(rec, gpart);
}

}  // namespace LBM_VARIANT
}  // namespace lbm
