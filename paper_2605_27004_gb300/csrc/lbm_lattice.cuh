// Compile-time velocity sets of the library: D2Q9, D3Q19, D3Q27 (Appendix C of the paper:
// tensor products of the D1Q3 Gauss-Hermite rule for D2Q9/D3Q27, the symmetry-reduced D3Q19).
//
// Direction order: 0 is the rest velocity; directions 2k+1 and 2k+2 are the pair +v_k, -v_k,
// so opp(i) = i + 1 for odd i and i - 1 for even i > 0. The positive half-vectors v_k are
//   axes      (1,0,0) (0,1,0) (0,0,1)
//   edges     (1,1,0) (1,-1,0) (1,0,1) (1,0,-1) (0,1,1) (0,1,-1)
//   corners   (1,1,1) (1,1,-1) (1,-1,1) (1,-1,-1)
// D2Q9 uses axes x, y and the two xy edges; D3Q19 axes + edges; D3Q27 all 13.
// Weights depend on |c|^2 only: D2Q9 4/9, 1/9, 1/36; D3Q19 1/3, 1/18, 1/36;
// D3Q27 8/27, 2/27, 1/54, 1/216.
#pragma once

namespace lbm {

struct Vec3 {
    int x, y, z;
};

__host__ __device__ constexpr Vec3 half_vec3(int k) {
    return k == 0    ? Vec3{1, 0, 0}
           : k == 1  ? Vec3{0, 1, 0}
           : k == 2  ? Vec3{0, 0, 1}
           : k == 3  ? Vec3{1, 1, 0}
           : k == 4  ? Vec3{1, -1, 0}
           : k == 5  ? Vec3{1, 0, 1}
           : k == 6  ? Vec3{1, 0, -1}
           : k == 7  ? Vec3{0, 1, 1}
           : k == 8  ? Vec3{0, 1, -1}
           : k == 9  ? Vec3{1, 1, 1}
           : k == 10 ? Vec3{1, 1, -1}
           : k == 11 ? Vec3{1, -1, 1}
                     : Vec3{1, -1, -1};
}

__host__ __device__ constexpr Vec3 half_vec2(int k) {
    return k == 0 ? Vec3{1, 0, 0} : k == 1 ? Vec3{0, 1, 0} : k == 2 ? Vec3{1, 1, 0} : Vec3{1, -1, 0};
}

template <int Q>
struct Lat;

template <>
struct Lat<9> {
    static constexpr int D = 2;
    static constexpr int P = 4;  // pairs
};
template <>
struct Lat<19> {
    static constexpr int D = 3;
    static constexpr int P = 9;
};
template <>
struct Lat<27> {
    static constexpr int D = 3;
    static constexpr int P = 13;
};

template <int Q>
__host__ __device__ constexpr Vec3 vel(int i) {
    // i = 0 rest; i = 2k+1 -> +v_k; i = 2k+2 -> -v_k
    return i == 0 ? Vec3{0, 0, 0}
                  : ((i & 1) ? (Q == 9 ? half_vec2((i - 1) / 2) : half_vec3((i - 1) / 2))
                             : Vec3{-(Q == 9 ? half_vec2((i - 2) / 2) : half_vec3((i - 2) / 2)).x,
                                    -(Q == 9 ? half_vec2((i - 2) / 2) : half_vec3((i - 2) / 2)).y,
                                    -(Q == 9 ? half_vec2((i - 2) / 2) : half_vec3((i - 2) / 2)).z});
}

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

template <int Q>
__host__ __device__ constexpr double weight(int i) {
    // |c|^2 classes
    return Q == 9 ? (vel<Q>(i).x * vel<Q>(i).x + vel<Q>(i).y * vel<Q>(i).y == 0   ? 4.0 / 9.0
                     : vel<Q>(i).x * vel<Q>(i).x + vel<Q>(i).y * vel<Q>(i).y == 1 ? 1.0 / 9.0
                                                                                    : 1.0 / 36.0)
           : Q == 19
               ? (vel<Q>(i).x * vel<Q>(i).x + vel<Q>(i).y * vel<Q>(i).y + vel<Q>(i).z * vel<Q>(i).z == 0 ? 1.0 / 3.0
                  : vel<Q>(i).x * vel<Q>(i).x + vel<Q>(i).y * vel<Q>(i).y + vel<Q>(i).z * vel<Q>(i).z == 1
                      ? 1.0 / 18.0
                      : 1.0 / 36.0)
               : (vel<Q>(i).x * vel<Q>(i).x + vel<Q>(i).y * vel<Q>(i).y + vel<Q>(i).z * vel<Q>(i).z == 0 ? 8.0 / 27.0
                  : vel<Q>(i).x * vel<Q>(i).x + vel<Q>(i).y * vel<Q>(i).y + vel<Q>(i).z * vel<Q>(i).z == 1
                      ? 2.0 / 27.0
                  : vel<Q>(i).x * vel<Q>(i).x + vel<Q>(i).y * vel<Q>(i).y + vel<Q>(i).z * vel<Q>(i).z == 2
                      ? 1.0 / 54.0
                      : 1.0 / 216.0);
}

}  // namespace lbm
