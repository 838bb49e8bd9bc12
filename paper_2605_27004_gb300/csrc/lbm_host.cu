// C-ABI implementation of include/lbm.h: context management, parameter validation, FP64 tables,
// the time-step loop (optionally replayed as CUDA graphs), observables, FP64 totals and the
// checkpointed discrete adjoint. Every numerical step runs in the kernels of lbm_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "lbm_lattice.cuh"

namespace lbm {

Shape shape_for(const Geom& g, int nzp) {
    Shape s;
    const int bx = block_x_for(g.nx);
    const int by = std::max(1, 256 / bx);
    s.block = dim3(bx, by, 1);
    s.grid = dim3((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, nzp);
    s.nblocks = (long long)s.grid.x * s.grid.y * s.grid.z;
    return s;
}

// Fixed-order FP64 sum: thread t adds records t, t + 1024, ... in order, then a fixed tree.
__global__ void __launch_bounds__(1024) k_reduce_partials(const double* __restrict__ part, long long nb, int width,
                                                          double* __restrict__ out) {
    __shared__ double sh[1024];
    for (int k = 0; k < width; ++k) {
        double s = 0.0;
        for (long long b = threadIdx.x; b < nb; b += blockDim.x) s += part[b * width + k];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

cudaError_t reduce_partials(const double* partials, long long nb, int width, double* out, cudaStream_t s) {
    k_reduce_partials<<<1, 1024, 0, s>>>(partials, nb, width, out);
    return cudaGetLastError();
}

// Halo planes of a z-slab: the directions dir[0..n-1] of stored plane `plane` of a [q][N] array,
// packed as [n][P] (P = nx*ny) into or out of a contiguous buffer.
struct HaloDirs {
    int n;
    int dir[9];
};

template <typename E>
__global__ void __launch_bounds__(256) k_halo_copy(E* __restrict__ arr, E* __restrict__ buf, HaloDirs hd, long long N,
                                                   long long P, long long plane, int pack) {
    const long long total = (long long)hd.n * P;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / P);
        E* a = arr + (long long)hd.dir[k] * N + plane * P + (t - (long long)k * P);
        if (pack)
            buf[t] = *a;
        else
            *a = buf[t];
    }
}

template <typename T>
__global__ void k_fill(T* __restrict__ p, long long n, T v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

static const Ops* ops_get(int q, int storage, bool slab) {
#define LBM_PICK(Q, SUF)                         \
    switch (storage) {                           \
        case 0: return &ops_q##Q##_s0##SUF();    \
        case 1: return &ops_q##Q##_s1##SUF();    \
        case 2: return &ops_q##Q##_s2##SUF();    \
        case 3: return &ops_q##Q##_s3##SUF();    \
        case 4: return &ops_q##Q##_s4##SUF();    \
        default: return nullptr;                 \
    }
    if (slab) {  // z-slab objects exist for the 3D lattices
        if (q == 19) LBM_PICK(19, _slab)
        if (q == 27) LBM_PICK(27, _slab)
        return nullptr;
    }
    if (q == 9) LBM_PICK(9, )
    if (q == 19) LBM_PICK(19, )
    if (q == 27) LBM_PICK(27, )
#undef LBM_PICK
    return nullptr;
}

template <int Q>
static Vec3 hvel(int i) {
    return vel<Q>(i);
}
template <int Q>
static double hweight(int i) {
    return weight<Q>(i);
}
static Vec3 velq(int q, int i) { return q == 9 ? hvel<9>(i) : q == 19 ? hvel<19>(i) : hvel<27>(i); }
static double weightq(int q, int i) { return q == 9 ? hweight<9>(i) : q == 19 ? hweight<19>(i) : hweight<27>(i); }

}  // namespace lbm

using namespace lbm;

struct lbm_ctx {
    int kind = 0;  // 0: flow (lbm_create), 1: advection-diffusion of a scalar (lbm_ade_create)
    int q = 0, d = 0, nx = 0, ny = 0, nz = 0;
    long long N = 0;
    double tau = 0.0;
    double Theta[9] = {0};
    lbm_options opt{};
    int storage = 0, scheme = 0, order = 3;
    size_t elem = 4;   // bytes per stored population
    size_t felem = 4;  // bytes per field value (float or double)
    const Ops* ops = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;

    Geom geom{};
    Shape shape{};
    uint32_t* link = nullptr;  // per-cell link words (N), null for an all-fluid box
    long long n_fluid = 0;
    uint32_t* cell_idx = nullptr;  // with walls: fluid cells (FP16 AA) or 32-byte sectors (FP16 / FP32 pull)
    CellList cells{};

    Coef<double> cd{};
    Coef<float> cf{};

    void* pop[2] = {nullptr, nullptr};
    int cur = 0;          // pull scheme: buffer holding the current state
    long long steps = 0;  // steps since init
    bool state_valid = false;
    bool init_fields = false;  // rho0/u0 copies are present for the adjoint
    void* rho_init = nullptr;
    void* u_init = nullptr;
    bool rho_init_null = true, u_init_null = true;

    int* flag = nullptr;
    double* partials = nullptr;  // nblocks * 8
    double* dout = nullptr;      // 8 doubles
    double* hout = nullptr;      // pinned 8 doubles
    int* hflag = nullptr;        // pinned

    // adjoint
    void* lam[2] = {nullptr, nullptr};
    void* du0 = nullptr;
    double* gpart = nullptr;
    bool grads_ready = false;
    int last_adj_K2 = 0;  // sub-segment length of the last adjoint (== K when flat)
    int last_adj_prefetch = 0;       // host checkpoints the last adjoint restored ahead of use
    std::vector<void*> adj_bufs;     // segment state buffers, kept for later adjoint calls
    double grad_theta[6] = {0};
    double grad_tau = 0.0;

    // advection-diffusion: library-owned advecting velocity [d][N] (field type), used unless zero
    void* ade_u = nullptr;
    bool ade_u_zero = true;

    // z-slab: ghost planes 0 and nz + 1 around nz interior planes (geom.z0 = 1)
    bool slab = false;
    void* halo_scratch = nullptr;  // two packed planes for the exchange of a slab with itself
    size_t halo_scratch_bytes = 0;

    // graphs
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;

    // checkpoints recorded during the forward run (state at t = k * rec_K)
    int rec_K = 0;
    std::vector<void*> rec_ptr;
    std::vector<bool> rec_host;
    long long rec_valid = 0;  // checkpoints 0 .. rec_valid-1 hold the current trajectory

    size_t dev_bytes = 0;
    long long launches = 0;
    std::string err;

    const void* coef() const { return storage == LBM_FP64 ? (const void*)&cd : (const void*)&cf; }
    size_t state_bytes() const { return (size_t)q * (size_t)N * elem; }
};

namespace {

int fail(lbm_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LBM_CUDA(ctx, call)                                       \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

void* dev_alloc(lbm_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (c->opt.alloc) {
        p = c->opt.alloc(bytes, c->opt.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        p = nullptr;
    }
    if (p) c->dev_bytes += bytes;
    return p;
}

void dev_free(lbm_ctx* c, void* p, size_t bytes) {
    if (!p) return;
    if (c->opt.alloc)
        c->opt.free(p, c->opt.alloc_user);
    else
        cudaFree(p);
    c->dev_bytes -= bytes;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Symmetric positive definite check by FP64 Cholesky.
int check_theta(lbm_ctx* c, int d, const double* Th) {
    if (!Th) return fail(c, LBM_ERR_INVALID_ARG, "Theta is NULL");
    double scale = 0.0;
    for (int k = 0; k < d * d; ++k) {
        if (!std::isfinite(Th[k])) return fail(c, LBM_ERR_INVALID_ARG, "Theta has a non-finite entry");
        scale = std::max(scale, std::fabs(Th[k]));
    }
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < a; ++b)
            if (std::fabs(Th[a * d + b] - Th[b * d + a]) > 1e-12 * std::max(1.0, scale))
                return fail(c, LBM_ERR_NOT_SPD, "Theta is not symmetric");
    double L[3][3] = {{0}};
    for (int i = 0; i < d; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = Th[i * d + j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0)) return fail(c, LBM_ERR_NOT_SPD, "Theta is not positive definite");
                L[i][i] = std::sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    return LBM_OK;
}

// FP64 coefficient tables for (tau, Theta, rho0, order), then one rounding to FP32.
void build_coef(lbm_ctx* c) {
    const int q = c->q, d = c->d;
    const double cs2 = 1.0 / 3.0;
    double Kt[3][3] = {{0}};
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Kt[a][b] = c->Theta[a * d + b] - (a == b ? cs2 : 0.0);
    double trK = 0.0;
    for (int a = 0; a < d; ++a) trK += Kt[a][a];
    Coef<double>& C = c->cd;
    std::memset(&C, 0, sizeof(C));
    const double rho0 = c->opt.rho0;
    C.omega = 1.0 / c->tau;
    C.rho0 = rho0;
    C.c3 = c->order == 3 ? 4.5 : 0.0;
    C.K[0] = Kt[0][0];
    C.K[1] = Kt[1][1];
    C.K[2] = Kt[2][2];
    C.K[3] = Kt[0][1];
    C.K[4] = Kt[0][2];
    C.K[5] = Kt[1][2];
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int i = 0; i < q; ++i) {
        const Vec3 v = velq(q, i);
        const double cv[3] = {(double)v.x, (double)v.y, (double)v.z};
        double h = -cs2 * trK;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) h += cv[a] * Kt[a][b] * cv[b];
        const double w = weightq(q, i);
        C.h[i] = h;
        C.A[i] = w * (1.0 + 4.5 * h);
        C.r[i] = rho0 * C.A[i];
        C.so[i] = c->storage == LBM_FP16_WSHIFTED ? C.r[i] - w * rho0
                  : (c->storage == LBM_FP32 || c->storage == LBM_FP64) ? C.r[i] : 0.0;
        C.B[i] = w * (3.0 + 3.0 * C.c3 * h);
        for (int k = 0; k < 6; ++k) C.Pirest[k] += C.r[i] * cv[pa[k]] * cv[pb[k]];
    }
    Coef<float>& F = c->cf;
    F.omega = (float)C.omega;
    F.rho0 = (float)C.rho0;
    F.c3 = (float)C.c3;
    for (int k = 0; k < 6; ++k) {
        F.K[k] = (float)C.K[k];
        F.Pirest[k] = (float)C.Pirest[k];
    }
    for (int i = 0; i < 27; ++i) {
        F.r[i] = (float)C.r[i];
        F.so[i] = (float)C.so[i];
        F.A[i] = (float)C.A[i];
        F.B[i] = (float)C.B[i];
        F.h[i] = (float)C.h[i];
    }
}

void drop_graph(lbm_ctx* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_steps = 0;
}

// One forward step src -> dst of a flow context on stream s (t = steps done before it): over the
// lists of a context with walls (sectors for pull, cells for FP16 AA), else over the grid.
cudaError_t step_kernel(lbm_ctx* c, const void* src, void* dst, long long t, cudaStream_t s) {
    if (c->cell_idx)
        return c->scheme == LBM_PULL2
                   ? c->ops->step_pull_sectors(c->geom, c->coef(), c->cells, src, dst, c->flag, s)
                   : c->ops->step_aa_list(c->geom, c->coef(), c->cells, (int)(t & 1), src, dst, c->flag, s);
    return c->scheme == LBM_PULL2 ? c->ops->step_pull(c->geom, c->coef(), src, dst, c->flag, s)
                                  : c->ops->step_aa(c->geom, c->coef(), (int)(t & 1), src, dst, c->flag, s);
}

int layout_now(const lbm_ctx* c, long long steps) {
    if (c->scheme == LBM_PULL2) return LAYOUT_PULL;
    return (steps & 1) ? LAYOUT_AAODD : LAYOUT_LOCAL;
}

void* state_ptr(lbm_ctx* c) { return c->scheme == LBM_PULL2 ? c->pop[c->cur] : c->pop[0]; }

// One time step from the current state, on stream s. Advances cur/steps.
cudaError_t launch_step(lbm_ctx* c, cudaStream_t s) {
    cudaError_t e;
    if (c->kind == 1) {
        const void* u = c->ade_u_zero ? nullptr : c->ade_u;
        if (c->scheme == LBM_PULL2) {
            e = c->cell_idx ? c->ops->ade_pull_sectors(c->geom, c->coef(), c->cells, u, c->pop[c->cur],
                                                       c->pop[c->cur ^ 1], c->flag, s)
                            : c->ops->ade_pull(c->geom, c->coef(), u, c->pop[c->cur], c->pop[c->cur ^ 1], c->flag, s);
            c->cur ^= 1;
        } else {
            e = c->ops->ade_aa(c->geom, c->coef(), u, (int)(c->steps & 1), c->pop[0], c->pop[0], c->flag, s);
        }
    } else if (c->scheme == LBM_PULL2) {
        e = step_kernel(c, c->pop[c->cur], c->pop[c->cur ^ 1], c->steps, s);
        c->cur ^= 1;
    } else {
        e = step_kernel(c, c->pop[0], c->pop[0], c->steps, s);
    }
    c->steps += 1;
    c->launches += 1;
    return e;
}

int ensure_graph(lbm_ctx* c, int gsteps) {
    if (c->graph && c->graph_steps == gsteps) return LBM_OK;
    drop_graph(c);
    if (!c->cap_stream) LBM_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const int cur0 = c->cur;
    const long long steps0 = c->steps;
    const long long launches0 = c->launches;
    LBM_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < gsteps && le == cudaSuccess; ++k) le = launch_step(c, c->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
    c->cur = cur0;
    c->steps = steps0;
    c->launches = launches0;
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, le, "kernel launch during graph capture");
    }
    if (ee != cudaSuccess) return cuda_fail(c, ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        c->graph = nullptr;
        return cuda_fail(c, ie, "cudaGraphInstantiate");
    }
    c->graph_steps = gsteps;
    return LBM_OK;
}

// Checkpoint k of the recorded trajectory: device memory while the adjoint limit allows, else
// pinned host memory. Returns null on allocation failure.
void* ckpt_slot(lbm_ctx* c, size_t k, bool* host) {
    const size_t SB = c->state_bytes();
    if (k < c->rec_ptr.size() && c->rec_ptr[k]) {
        *host = c->rec_host[k];
        return c->rec_ptr[k];
    }
    if (c->rec_ptr.size() <= k) {
        c->rec_ptr.resize(k + 1, nullptr);
        c->rec_host.resize(k + 1, false);
    }
    // Device memory while the checkpoints stay within adjoint_mem_limit and leave room for the
    // adjoint's own working set (two lambda arrays, du0, and the smallest two-level segment
    // plan, 2 sqrt(K) states); pinned host memory beyond.
    size_t used = 0;
    for (size_t j = 0; j < c->rec_ptr.size(); ++j)
        if (c->rec_ptr[j] && !c->rec_host[j]) used += SB;
    size_t fr = 0, tot = 0;
    bool dev_ok = cudaMemGetInfo(&fr, &tot) == cudaSuccess;
    if (!dev_ok) (void)cudaGetLastError();
    const size_t LB = (size_t)c->q * c->N * c->felem;
    const long long plan = 2 * (long long)std::ceil(std::sqrt((double)c->rec_K)) + 1;  // states
    const long long to_get = std::max<long long>(0, plan - (long long)c->adj_bufs.size());
    const size_t reserve = (c->lam[0] ? 0 : 2 * LB + (size_t)c->d * c->N * c->felem) + (size_t)to_get * SB +
                           ((size_t)2 << 30);
    dev_ok = dev_ok && fr >= reserve + SB;
    if (c->opt.adjoint_mem_limit)  // the limit covers checkpoints and the smallest segment plan
        dev_ok = dev_ok && used + SB + (size_t)(2 * (int)std::ceil(std::sqrt((double)c->rec_K)) + 1) * SB <=
                               c->opt.adjoint_mem_limit;
    void* p = nullptr;
    bool h = false;
    if (dev_ok) p = dev_alloc(c, SB);
    if (!p) {
        if (cudaMallocHost(&p, SB) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        h = true;
    }
    c->rec_ptr[k] = p;
    c->rec_host[k] = h;
    *host = h;
    return p;
}

int record_ckpt(lbm_ctx* c) {
    if (c->rec_K <= 0 || c->steps % c->rec_K != 0) return LBM_OK;
    const long long k = c->steps / c->rec_K;
    if (k != c->rec_valid) return LBM_OK;  // only extend a contiguous record
    bool host = false;
    void* p = ckpt_slot(c, (size_t)k, &host);
    if (!p) return fail(c, LBM_ERR_OOM, "checkpoint %lld", k);
    LBM_CUDA(c, cudaMemcpyAsync(p, state_ptr(c), c->state_bytes(), cudaMemcpyDefault, c->stream));
    c->rec_valid = k + 1;
    return LBM_OK;
}

int check_flag(lbm_ctx* c) {
    LBM_CUDA(c, cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (*c->hflag)
        return fail(c, LBM_ERR_UNSTABLE, c->kind == 1 ? "a fluid cell reached a non-finite scalar"
                                                      : "a fluid cell reached rho <= 0 or a non-finite value");
    return LBM_OK;
}

int flow_only(lbm_ctx* c, const char* what) {
    return c->kind == 1 ? fail(c, LBM_ERR_INVALID_ARG, "%s: defined for flow contexts only", what) : LBM_OK;
}

// --- z-slab halo planes ----------------------------------------------------------------------
// c_z of the directions a pack on `side` carries: populations stream along +c_i, so the slab
// below needs the c_z = -1 populations of the lowest interior plane (side 0) and the slab above
// the c_z = +1 ones of the highest (side 1); lambda streams backwards, so the signs flip. An
// unpack into the ghost plane on `side` receives what the neighbour on that side packed for its
// opposite side.
int halo_sign(int kind, int pack_side) { return (kind == LBM_HALO_POPULATIONS) == (pack_side == 0) ? -1 : 1; }

HaloDirs halo_dirs(int q, int sign) {
    HaloDirs hd{};
    for (int i = 0; i < q; ++i)
        if (velq(q, i).z == sign) hd.dir[hd.n++] = i;
    return hd;
}

size_t halo_bytes_of(const lbm_ctx* c, int kind) {
    const size_t el = kind == LBM_HALO_POPULATIONS ? c->elem : c->felem;
    return (size_t)halo_dirs(c->q, 1).n * (size_t)c->nx * (size_t)c->ny * el;
}

cudaError_t halo_copy(lbm_ctx* c, int kind, int side, bool pack, void* array, void* buf) {
    const HaloDirs hd = halo_dirs(c->q, halo_sign(kind, pack ? side : 1 - side));
    const long long P = (long long)c->nx * c->ny;
    const long long plane = pack ? (side == 0 ? 1 : c->nz) : (side == 0 ? 0 : c->nz + 1);
    const size_t el = kind == LBM_HALO_POPULATIONS ? c->elem : c->felem;
    const long long total = (long long)hd.n * P;
    const unsigned nb = (unsigned)std::max<long long>(1, std::min<long long>((total + 255) / 256, 8 * 152));
    const int pk = pack ? 1 : 0;
    if (el == 2)
        k_halo_copy<uint16_t><<<nb, 256, 0, c->stream>>>((uint16_t*)array, (uint16_t*)buf, hd, c->N, P, plane, pk);
    else if (el == 4)
        k_halo_copy<uint32_t><<<nb, 256, 0, c->stream>>>((uint32_t*)array, (uint32_t*)buf, hd, c->N, P, plane, pk);
    else
        k_halo_copy<uint64_t><<<nb, 256, 0, c->stream>>>((uint64_t*)array, (uint64_t*)buf, hd, c->N, P, plane, pk);
    c->launches += 1;
    return cudaGetLastError();
}

// Fill the ghost planes of a [q][N] array that the last kernel wrote: through the caller's
// exchange callback, or, without one, from the slab's own boundary planes (the slab is then the
// whole box in z, periodic).
int run_halo(lbm_ctx* c, int kind, void* array) {
    if (!c->slab) return LBM_OK;
    if (c->opt.halo) {
        const int rc = c->opt.halo(c, kind, array, c->opt.halo_user);
        if (rc != 0) return fail(c, LBM_ERR_HALO, "halo exchange callback returned %d", rc);
        return LBM_OK;
    }
    char* s0 = (char*)c->halo_scratch;
    char* s1 = s0 + c->halo_scratch_bytes / 2;
    cudaError_t e = halo_copy(c, kind, 1, true, array, s0);  // top plane -> ghost below
    if (e == cudaSuccess) e = halo_copy(c, kind, 0, false, array, s0);
    if (e == cudaSuccess) e = halo_copy(c, kind, 0, true, array, s1);  // bottom plane -> ghost above
    if (e == cudaSuccess) e = halo_copy(c, kind, 1, false, array, s1);
    if (e != cudaSuccess) return cuda_fail(c, e, "halo copy");
    return LBM_OK;
}

// Recompute plan of one adjoint segment of `len` steps with W working state buffers. Flat
// (len - 1 <= W): all states after the segment start are recomputed once and held. Otherwise the
// segment is cut at starts 0 = s_0 < s_1 < ... < s_m < len: the first recompute pass keeps the
// states s_1 .. s_(m-1) and every state of the last sub-segment [s_m, len) (L = len - s_m
// buffers), which is swept first; each earlier sub-segment (at most L + 1 steps) is then
// recomputed from its start into the last one's buffers and swept. W = (m - 1) + L buffers, and
// the plan costs (len - 1) + (s_m - m) recompute steps, i.e. 2 len - 2 - W when m = W - L + 1:
// every buffer saves one step, whatever L. The largest feasible L (fewest sub-segments) is
// taken; L >= 2 so that the first pass can alternate two of the last sub-segment's buffers for
// the states it does not keep. Returns false when W buffers admit no such plan; on success
// `starts` holds s_0 .. s_m (just {0} when flat).
bool segment_plan(int len, int W, std::vector<int>& starts) {
    starts.assign(1, 0);
    if (len - 1 <= W) return true;
    for (int L = W; L >= 2; --L) {
        const int rest = len - L;        // steps before the last sub-segment
        const int m1 = W - L + 1;        // sub-segments the buffers allow before it
        if ((long long)m1 * (L + 1) < rest) continue;
        const int m = std::min(m1, rest);
        for (int j = 0, s = 0; j < m; ++j) {
            s += rest / m + (j < rest % m ? 1 : 0);
            starts.push_back(s);
        }
        return true;
    }
    return false;
}

}  // namespace

// =============================================================================================
extern "C" {

int lbm_options_default(lbm_options* opt) {
    if (!opt) return LBM_ERR_INVALID_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->storage = LBM_FP32_SHIFTED;
    opt->scheme = LBM_PULL2;
    opt->order = 3;
    opt->rho0 = 1.0;
    return LBM_OK;
}

const char* lbm_status_string(int s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_ERR_INVALID_ARG: return "invalid argument";
        case LBM_ERR_NOT_SPD: return "Theta is not symmetric positive definite";
        case LBM_ERR_BAD_TAU: return "tau must exceed 1/2";
        case LBM_ERR_OOM: return "out of memory";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_UNSTABLE: return "simulation became unstable";
        case LBM_ERR_NO_FORWARD: return "adjoint needs exactly n forward steps since lbm_init";
        case LBM_ERR_TIMEOUT: return "device wait timed out";
        case LBM_ERR_STATE: return "call out of order";
        case LBM_ERR_HALO: return "halo exchange callback failed";
        default: return "unknown status";
    }
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "no context"; }

int lbm_lattice_info(int lattice, int* c, double* w) {
    if (lattice != 9 && lattice != 19 && lattice != 27) return LBM_ERR_INVALID_ARG;
    for (int i = 0; i < lattice; ++i) {
        const Vec3 v = velq(lattice, i);
        if (c) {
            c[3 * i] = v.x;
            c[3 * i + 1] = v.y;
            c[3 * i + 2] = v.z;
        }
        if (w) w[i] = weightq(lattice, i);
    }
    return lattice;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graph(c);
    const size_t SB = c->state_bytes();
    dev_free(c, c->pop[0], SB);
    dev_free(c, c->pop[1], SB);
    dev_free(c, c->link, (size_t)c->N * 4);
    dev_free(c, c->cell_idx, (size_t)c->cells.count * 4 + 4);
    for (size_t k = 0; k < c->rec_ptr.size(); ++k) {
        if (!c->rec_ptr[k]) continue;
        if (c->rec_host[k])
            cudaFreeHost(c->rec_ptr[k]);
        else
            dev_free(c, c->rec_ptr[k], c->state_bytes());
    }
    dev_free(c, c->rho_init, (size_t)c->N * c->felem);
    dev_free(c, c->u_init, (size_t)c->N * c->d * c->felem);
    dev_free(c, c->flag, sizeof(int) * 2);
    dev_free(c, c->partials, (size_t)c->shape.nblocks * 8 * sizeof(double));
    dev_free(c, c->dout, 8 * sizeof(double));
    const size_t LB = (size_t)c->q * c->N * c->felem;
    dev_free(c, c->lam[0], LB);
    dev_free(c, c->lam[1], LB);
    dev_free(c, c->du0, (size_t)c->d * c->N * c->felem);
    dev_free(c, c->gpart, (size_t)c->shape.nblocks * 8 * sizeof(double));
    for (void* p : c->adj_bufs) dev_free(c, p, SB);
    dev_free(c, c->ade_u, (size_t)c->d * c->N * c->felem);
    dev_free(c, c->halo_scratch, c->halo_scratch_bytes);
    if (c->hout) cudaFreeHost(c->hout);
    if (c->hflag) cudaFreeHost(c->hflag);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

int lbm_create_ex(lbm_ctx** out, int lattice, int nx, int ny, int nz, double tau, const double* Theta,
                  const uint8_t* solid_mask, const lbm_options* opt) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_OOM;
    auto bail = [&](int code) {
        std::string keep = c->err;
        lbm_destroy(c);
        (void)keep;
        return code;
    };
    if (opt)
        c->opt = *opt;
    else
        lbm_options_default(&c->opt);
    if (c->opt.order == 0) c->opt.order = 3;
    if (c->opt.rho0 == 0.0) c->opt.rho0 = 1.0;
    if (lattice != 9 && lattice != 19 && lattice != 27) return bail(LBM_ERR_INVALID_ARG);
    if (c->opt.storage < 0 || c->opt.storage > 4 || c->opt.scheme < 0 || c->opt.scheme > 1) return bail(LBM_ERR_INVALID_ARG);
    if (c->opt.order != 2 && c->opt.order != 3) return bail(LBM_ERR_INVALID_ARG);
    if (!(c->opt.rho0 > 0.0) || !std::isfinite(c->opt.rho0)) return bail(LBM_ERR_INVALID_ARG);
    if ((c->opt.alloc == nullptr) != (c->opt.free == nullptr)) return bail(LBM_ERR_INVALID_ARG);
    c->q = lattice;
    c->d = lattice == 9 ? 2 : 3;
    if (nx < 1 || ny < 1 || nz < 1 || (c->d == 2 && nz != 1)) return bail(LBM_ERR_INVALID_ARG);
    c->slab = c->opt.z_halo != 0;
    if (c->slab && (c->d != 3 || c->opt.scheme != LBM_PULL2))
        return bail(fail(c, LBM_ERR_INVALID_ARG, "z-slab contexts need D3Q19/D3Q27 and the pull scheme"));
    if (!c->slab && c->opt.halo) return bail(fail(c, LBM_ERR_INVALID_ARG, "halo callback without z_halo"));
    const int nzs = c->slab ? nz + 2 : nz;  // stored planes
    {
        Geom g0{};
        g0.nx = nx;
        g0.ny = ny;
        g0.nz = nzs;
        const Shape s0 = shape_for(g0, nz);
        if (nz > 65535 || s0.grid.y > 65535u) return bail(LBM_ERR_INVALID_ARG);
    }
    if (!(tau > 0.5) || !std::isfinite(tau)) return bail(LBM_ERR_BAD_TAU);
    int rc = check_theta(c, c->d, Theta);
    if (rc) return bail(rc);
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->N = (long long)nx * ny * nzs;
    c->tau = tau;
    for (int k = 0; k < c->d * c->d; ++k) c->Theta[k] = Theta[k];
    c->storage = c->opt.storage;
    c->scheme = c->opt.scheme;
    c->order = c->opt.order;
    c->elem = c->storage == LBM_FP64 ? 8 : (c->storage == LBM_FP16_SHIFTED || c->storage == LBM_FP16_WSHIFTED) ? 2 : 4;
    c->felem = c->storage == LBM_FP64 ? 8 : 4;
    c->ops = ops_get(c->q, c->storage, c->slab);
    c->stream = (cudaStream_t)c->opt.stream;
    build_coef(c);

    if (c->N >= (1LL << 31)) return bail(fail(c, LBM_ERR_INVALID_ARG, "more than 2^31 - 1 cells"));
    c->geom.nx = nx;
    c->geom.ny = ny;
    c->geom.nz = nzs;
    c->geom.N = (uint32_t)c->N;
    c->geom.link = nullptr;
    c->shape = shape_for(c->geom, nz);
    const long long plane = (long long)nx * ny;
    c->n_fluid = plane * nz;  // interior cells

    if (solid_mask) {
        std::vector<uint8_t> m((size_t)c->N);
        const bool on_dev = is_device_ptr(solid_mask);
        if (on_dev) {
            if (cudaMemcpy(m.data(), solid_mask, (size_t)c->N, cudaMemcpyDeviceToHost) != cudaSuccess)
                return bail(cuda_fail(c, cudaGetLastError(), "copy of the solid mask"));
        } else {
            std::memcpy(m.data(), solid_mask, (size_t)c->N);
        }
        long long nsolid = 0, nsolid_int = 0;
        for (size_t n = 0; n < (size_t)c->N; ++n) {
            nsolid += m[n] != 0;
            if (!c->slab || ((long long)n >= plane && (long long)n < plane * (nz + 1))) nsolid_int += m[n] != 0;
        }
        c->n_fluid = plane * nz - nsolid_int;
        if (nsolid > 0) {
            c->link = (uint32_t*)dev_alloc(c, (size_t)c->N * 4);
            uint8_t* dmask = (uint8_t*)dev_alloc(c, (size_t)c->N);
            if (!c->link || !dmask) {
                dev_free(c, dmask, (size_t)c->N);
                return bail(fail(c, LBM_ERR_OOM, "link-mask allocation"));
            }
            cudaError_t e = cudaMemcpyAsync(dmask, m.data(), (size_t)c->N, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->link, 0, (size_t)c->N * 4, c->stream);  // ghost planes
            if (e == cudaSuccess) e = c->ops->link_mask(c->geom, dmask, c->link, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            dev_free(c, dmask, (size_t)c->N);
            if (e != cudaSuccess) return bail(cuda_fail(c, e, "link-mask construction"));
            c->geom.link = c->link;
            // Lists over the interior planes. FP16 storage is limited by issued instructions: the AA
            // steps run over the fluid cells (no lane of a warp belongs to a solid cell), the pull
            // step over the 32-byte sectors (16 cells) that hold a fluid cell (its stores stay whole
            // sectors). The D3Q27 FP32 pull step runs over its 8-cell sectors the same way, so that
            // no warp slot is spent on a sector of solid cells only (porous D3Q27 512^3: 0.714 ->
            // 0.750 of the copy peak on fluid accounting; the scalar at 256^3 0.706 -> 0.738); the
            // lighter D3Q19 FP32 cell update lost by it (scalar, 512^3: 0.708 -> 0.668) and stays on
            // the grid.
            const bool fp16 = c->storage == LBM_FP16_SHIFTED || c->storage == LBM_FP16_WSHIFTED;
            const bool fp32 = c->storage == LBM_FP32 || c->storage == LBM_FP32_SHIFTED;
            if ((fp16 || (fp32 && c->q == 27 && c->scheme == LBM_PULL2)) && nx >= 2) {
                std::vector<uint32_t> idx;
                const long long z0 = c->slab ? 1 : 0;
                const long long nb = z0 * plane, ne = (z0 + nz) * plane;
                if (c->scheme == LBM_AA) {
                    idx.reserve((size_t)c->n_fluid);
                    for (long long n = nb; n < ne; ++n)
                        if (!m[(size_t)n]) idx.push_back((uint32_t)n);
                } else {
                    const long long G = fp16 ? 16 : 8;  // cells of one 32-byte sector
                    for (long long s0 = nb / G; s0 * G < ne; ++s0) {
                        bool any = false;
                        for (long long n = std::max(s0 * G, nb); n < std::min(s0 * G + G, ne) && !any; ++n)
                            any = !m[(size_t)n];
                        if (any) idx.push_back((uint32_t)s0);
                    }
                }
                c->cell_idx = (uint32_t*)dev_alloc(c, idx.size() * 4 + 4);
                if (!c->cell_idx) return bail(fail(c, LBM_ERR_OOM, "fluid-cell list"));
                e = cudaMemcpy(c->cell_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice);
                if (e != cudaSuccess) return bail(cuda_fail(c, e, "fluid-cell list upload"));
                c->cells.idx = c->cell_idx;
                c->cells.count = (uint32_t)idx.size();
                c->cells.rnx = ~0ULL / (unsigned long long)nx + 1ULL;
                c->cells.rnxy = ~0ULL / (unsigned long long)plane + 1ULL;
                c->cells.n_begin = (uint32_t)nb;
                c->cells.n_end = (uint32_t)ne;
            }
        }
    }
    const size_t SB = c->state_bytes();
    c->pop[0] = dev_alloc(c, SB);
    if (c->scheme == LBM_PULL2) c->pop[1] = dev_alloc(c, SB);
    c->flag = (int*)dev_alloc(c, sizeof(int) * 2);
    if (c->slab) {
        c->halo_scratch_bytes = 2 * std::max(halo_bytes_of(c, LBM_HALO_POPULATIONS), halo_bytes_of(c, LBM_HALO_ADJOINT));
        c->halo_scratch = dev_alloc(c, c->halo_scratch_bytes);
        if (!c->halo_scratch) return bail(fail(c, LBM_ERR_OOM, "halo buffers"));
    }
    c->partials = (double*)dev_alloc(c, (size_t)c->shape.nblocks * 8 * sizeof(double));
    c->dout = (double*)dev_alloc(c, 8 * sizeof(double));
    if (!c->pop[0] || (c->scheme == LBM_PULL2 && !c->pop[1]) || !c->flag || !c->partials || !c->dout)
        return bail(fail(c, LBM_ERR_OOM, "population allocation (%zu bytes per array)", SB));
    if (cudaMallocHost(&c->hout, 8 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->hflag, 2 * sizeof(int)) != cudaSuccess)
        return bail(fail(c, LBM_ERR_OOM, "pinned host allocation"));
    // solid-cell slots are never written by the kernels; keep them defined
    if (cudaMemsetAsync(c->pop[0], 0, SB, c->stream) != cudaSuccess ||
        (c->pop[1] && cudaMemsetAsync(c->pop[1], 0, SB, c->stream) != cudaSuccess) ||
        cudaMemsetAsync(c->flag, 0, sizeof(int) * 2, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return bail(cuda_fail(c, cudaGetLastError(), "buffer clear"));
    *out = c;
    return LBM_OK;
}

int lbm_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, double tau, const double* Theta,
               const uint8_t* solid_mask) {
    return lbm_create_ex(out, lattice, nx, ny, nz, tau, Theta, solid_mask, nullptr);
}

int lbm_set_params(lbm_ctx* c, double tau, const double* Theta) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(c, LBM_ERR_BAD_TAU, "tau = %g", tau);
    int rc = check_theta(c, c->d, Theta);
    if (rc) return rc;
    c->tau = tau;
    for (int k = 0; k < c->d * c->d; ++k) c->Theta[k] = Theta[k];
    build_coef(c);
    drop_graph(c);
    c->state_valid = false;
    c->init_fields = false;
    c->grads_ready = false;
    c->rec_valid = 0;
    return LBM_OK;
}

int lbm_init(lbm_ctx* c, const void* rho, const void* u) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (c->kind == 1 && u)
        return fail(c, LBM_ERR_INVALID_ARG, "lbm_init of a scalar context takes u = NULL (the advecting velocity)");
    const size_t FN = (size_t)c->N * c->felem;
    if (!c->rho_init) c->rho_init = dev_alloc(c, FN);
    if (!c->u_init) c->u_init = dev_alloc(c, FN * c->d);
    if (!c->rho_init || !c->u_init) return fail(c, LBM_ERR_OOM, "initial-field copies");
    if (rho) LBM_CUDA(c, cudaMemcpyAsync(c->rho_init, rho, FN, cudaMemcpyDefault, c->stream));
    if (u) LBM_CUDA(c, cudaMemcpyAsync(c->u_init, u, FN * c->d, cudaMemcpyDefault, c->stream));
    c->rho_init_null = rho == nullptr;
    c->u_init_null = u == nullptr;
    c->cur = 0;
    c->steps = 0;
    const int layout = c->scheme == LBM_PULL2 ? LAYOUT_PULL : LAYOUT_LOCAL;
    const void* ui = u ? c->u_init : (c->kind == 1 && !c->ade_u_zero ? c->ade_u : nullptr);
    cudaError_t e = c->ops->init(c->geom, c->coef(), layout, rho ? c->rho_init : nullptr, ui, c->pop[0], c->stream);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    LBM_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    c->state_valid = true;
    c->init_fields = true;
    c->grads_ready = false;
    c->rec_valid = 0;
    return record_ckpt(c);
}

int lbm_record_checkpoints(lbm_ctx* c, int checkpoint_every) {
    if (!c || checkpoint_every < 0) return LBM_ERR_INVALID_ARG;
    if (int rc = flow_only(c, "lbm_record_checkpoints")) return rc;
    c->rec_K = checkpoint_every;
    c->rec_valid = 0;
    if (checkpoint_every > 0 && c->state_valid && c->steps == 0 && c->init_fields) return record_ckpt(c);
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
    if (!c || n < 0) return LBM_ERR_INVALID_ARG;
    if (!c->state_valid) return fail(c, LBM_ERR_STATE, "lbm_step before lbm_init");
    const int gsteps = 16;
    bool graphs = !c->slab && (c->opt.use_graphs > 0 || (c->opt.use_graphs == 0 && c->N <= (1LL << 21)));
    long long next_check = c->opt.check_every > 0 ? (c->steps / c->opt.check_every + 1) * c->opt.check_every : -1;
    const bool recording = c->rec_K > 0 && c->rec_valid * c->rec_K > c->steps;
    long long next_rec = recording ? (c->steps / c->rec_K + 1) * c->rec_K : -1;
    int left = n;
    while (left > 0) {
        const bool aligned = (c->steps & 1) == 0 && (c->scheme != LBM_PULL2 || c->cur == 0);
        bool ran = false;
        if (graphs && left >= gsteps && aligned && (next_check < 0 || c->steps + gsteps <= next_check) &&
            (next_rec < 0 || c->steps + gsteps <= next_rec)) {
            int rc = ensure_graph(c, gsteps);
            if (rc) return rc;
            LBM_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
            c->steps += gsteps;
            c->launches += gsteps;
            left -= gsteps;
            ran = true;
        }
        if (!ran) {
            cudaError_t e = launch_step(c, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "stream-collide kernel");
            if (int rc = run_halo(c, LBM_HALO_POPULATIONS, state_ptr(c))) return rc;
            left -= 1;
        }
        if (next_check >= 0 && c->steps >= next_check) {
            int rc = check_flag(c);
            if (rc) return rc;
            next_check += c->opt.check_every;
        }
        if (next_rec >= 0 && c->steps >= next_rec) {
            int rc = record_ckpt(c);
            if (rc) return rc;
            next_rec += c->rec_K;
        }
    }
    return LBM_OK;
}

int lbm_moments(lbm_ctx* c, void* rho, void* u, void* Pi) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!c->state_valid) return fail(c, LBM_ERR_STATE, "lbm_moments before lbm_init");
    if (!rho && !u && !Pi) return LBM_OK;
    cudaError_t e = c->ops->moments(c->geom, c->coef(), layout_now(c, c->steps), state_ptr(c), rho, u, Pi, nullptr,
                                    c->stream);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
    return LBM_OK;
}

int lbm_populations(lbm_ctx* c, void* f) {
    if (!c || !f) return LBM_ERR_INVALID_ARG;
    if (!c->state_valid) return fail(c, LBM_ERR_STATE, "lbm_populations before lbm_init");
    cudaError_t e = c->ops->moments(c->geom, c->coef(), layout_now(c, c->steps), state_ptr(c), nullptr, nullptr,
                                    nullptr, f, c->stream);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, "populations kernel");
    return LBM_OK;
}

int lbm_totals(lbm_ctx* c, double* mass, double* momentum) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!c->state_valid) return fail(c, LBM_ERR_STATE, "lbm_totals before lbm_init");
    LBM_CUDA(c, cudaMemsetAsync(c->flag + 1, 0, sizeof(int), c->stream));
    cudaError_t e = c->ops->totals(c->geom, c->coef(), layout_now(c, c->steps), state_ptr(c), c->partials,
                                   c->flag + 1, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "totals kernel");
    e = reduce_partials(c->partials, c->shape.nblocks, 4, c->dout, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "totals reduction");
    c->launches += 2;
    LBM_CUDA(c, cudaMemcpyAsync(c->hout, c->dout, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(c->hflag + 1, c->flag + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (mass) *mass = c->hout[0];
    if (momentum)
        for (int a = 0; a < c->d; ++a) momentum[a] = c->hout[1 + a];
    if (c->kind == 1) {  // a scalar may be zero or negative; only non-finite values are failures
        for (int a = 0; a <= c->d; ++a)
            if (!std::isfinite(c->hout[a])) return fail(c, LBM_ERR_UNSTABLE, "a non-finite scalar total");
        return LBM_OK;
    }
    if (c->hflag[1]) return fail(c, LBM_ERR_UNSTABLE, "a fluid cell has rho <= 0 or a non-finite moment");
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------------
// Discrete adjoint with checkpointing. States are kept in the stored form, so a recomputed
// state is bit-identical to the forward one.
// ---------------------------------------------------------------------------------------------
int lbm_adjoint(lbm_ctx* c, const void* loss_grad, int n, int K) {
    if (!c || !loss_grad || n < 0 || K < 0) return LBM_ERR_INVALID_ARG;
    if (int rc = flow_only(c, "lbm_adjoint")) return rc;
    if (!c->init_fields || !c->state_valid || c->steps != n)
        return fail(c, LBM_ERR_NO_FORWARD, "adjoint over %d steps but %lld steps were run since lbm_init", n,
                    (long long)c->steps);
    if (K == 0) K = c->rec_K > 0 ? c->rec_K : std::max(1, (int)std::lround(std::sqrt((double)std::max(n, 1))));
    K = std::max(1, std::min(K, std::max(n, 1)));
    const size_t SB = c->state_bytes();
    const size_t LB = (size_t)c->q * c->N * c->felem;
    const size_t GB = (size_t)c->shape.nblocks * 8 * sizeof(double);
    if (!c->lam[0]) {
        c->lam[0] = dev_alloc(c, LB);
        c->lam[1] = dev_alloc(c, LB);
        c->du0 = dev_alloc(c, (size_t)c->d * c->N * c->felem);
        c->gpart = (double*)dev_alloc(c, GB);
        if (!c->lam[0] || !c->lam[1] || !c->du0 || !c->gpart) return fail(c, LBM_ERR_OOM, "adjoint buffers");
        LBM_CUDA(c, cudaMemsetAsync(c->lam[0], 0, LB, c->stream));
        LBM_CUDA(c, cudaMemsetAsync(c->lam[1], 0, LB, c->stream));
    }
    LBM_CUDA(c, cudaMemsetAsync(c->gpart, 0, GB, c->stream));
    c->grads_ready = false;

    const int C = (n + K - 1) / K;  // top-level checkpoints at t = 0, K, ..., (C-1)K
    const bool recorded = c->rec_K == K && c->rec_valid >= C;

    // Memory plan for the states of one segment (segment_plan), next to bufs[0], the restore
    // target of host checkpoints: flat when the K - 1 states fit; else, while the checkpoints are
    // still to be taken, the fewest working buffers that admit a plan (device memory left to the
    // checkpoints saves copies to and from the host), and over recorded checkpoints every buffer
    // that fits, less one kept for restoring host checkpoints a segment ahead of use. Segment
    // buffers are kept in the context for later calls, so they count as available.
    size_t fr = 0, tot = 0;
    LBM_CUDA(c, cudaMemGetInfo(&fr, &tot));
    const long long held = (long long)c->adj_bufs.size();
    size_t avail = (fr > ((size_t)1 << 30) ? fr - ((size_t)1 << 30) : 0) + (size_t)held * SB;
    if (c->opt.adjoint_mem_limit) avail = std::min(avail, c->opt.adjoint_mem_limit);
    const long long mbuf = (long long)(avail / SB);
    int W = K - 1;  // working state buffers besides bufs[0]
    if (K > mbuf) {
        int wmin = -1;
        std::vector<int> sp;
        for (int w = 2; w < K - 1 && wmin < 0; ++w)
            if (segment_plan(K, w, sp)) wmin = w;
        if (wmin < 0 || wmin + 1 > mbuf)
            return fail(c, LBM_ERR_OOM, "adjoint: segment of %d steps needs %d states of %zu bytes, %lld fit", K,
                        wmin < 0 ? K : wmin + 1, SB, mbuf);
        W = wmin;
        if (recorded) {
            int n_dev = 0, n_host = 0;
            for (int k = 0; k < C; ++k) (c->rec_host[k] ? n_host : n_dev) += 1;
            long long budget = mbuf;  // the limit also covers the recorded device checkpoints
            if (c->opt.adjoint_mem_limit)
                budget = std::min<long long>(budget, (long long)(c->opt.adjoint_mem_limit / SB) - n_dev);
            W = (int)std::max<long long>(wmin, std::min<long long>(K - 2, budget - 1 - (n_host > 1 ? 1 : 0)));
        }
    }
    const bool flat_plan = W >= K - 1;
    const int nbuf = std::max(2, W + 1);
    int longest = K;  // longest sub-segment of a full segment, reported by lbm_adjoint_info
    if (!flat_plan) {
        std::vector<int> sp;
        segment_plan(K, W, sp);
        longest = K - sp.back();
        for (size_t j = 0; j + 1 < sp.size(); ++j) longest = std::max(longest, sp[j + 1] - sp[j]);
    }

    std::vector<void*> ckpt(C, nullptr);
    std::vector<bool> ckpt_host(C, false);
    std::vector<void*> own;  // checkpoints this call allocated
    std::vector<bool> own_host;
    cudaStream_t cs = nullptr;  // copy stream of the checkpoint prefetch
    cudaEvent_t ev_free = nullptr, ev_done[2] = {nullptr, nullptr};
    cudaGraphExec_t seg_graph = nullptr;  // one full segment, replayed (small boxes)
    auto release = [&]() {
        cudaStreamSynchronize(c->stream);
        if (seg_graph) cudaGraphExecDestroy(seg_graph);
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        for (cudaEvent_t e : {ev_free, ev_done[0], ev_done[1]})
            if (e) cudaEventDestroy(e);
        for (size_t k = 0; k < own.size(); ++k) {
            if (own_host[k])
                cudaFreeHost(own[k]);
            else
                dev_free(c, own[k], SB);
        }
    };
    int rc = LBM_OK;
#define LBM_ADJ_CHECK(expr, what)          \
    do {                                   \
        cudaError_t e_ = (expr);           \
        if (e_ != cudaSuccess) {           \
            rc = cuda_fail(c, e_, what);   \
            release();                     \
            return rc;                     \
        }                                  \
    } while (0)
    for (long long k = held; k < nbuf; ++k) {
        void* p = dev_alloc(c, SB);
        if (!p) return fail(c, LBM_ERR_OOM, "adjoint: segment state %lld of %d (%zu bytes)", k, nbuf, SB);
        c->adj_bufs.push_back(p);
        // solid-cell slots that no kernel writes stay defined
        LBM_CUDA(c, cudaMemsetAsync(p, 0, SB, c->stream));
    }
    void** bufs = c->adj_bufs.data();
    const void* cf = c->coef();
    // one forward step src -> dst (then the ghost planes of dst, for a z-slab)
    auto step_oop = [&](const void* src, void* dst, long long t, const char* what) -> int {
        c->launches += 1;
        const cudaError_t e = step_kernel(c, src, dst, t, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, what);
        return run_halo(c, LBM_HALO_POPULATIONS, dst);
    };
#define LBM_ADJ_RC(expr)              \
    do {                              \
        const int r_ = (expr);        \
        if (r_ != LBM_OK) {           \
            release();                \
            return r_;                \
        }                             \
    } while (0)

    if (recorded) {
        for (int k = 0; k < C; ++k) {
            ckpt[k] = c->rec_ptr[k];
            ckpt_host[k] = c->rec_host[k];
        }
    } else {
        // Forward pass from the initial fields, keeping the state at multiples of K (device while
        // it fits next to the segment buffers, pinned host memory beyond).
        LBM_ADJ_CHECK(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
        long long room = (long long)(fr > ((size_t)1 << 30) ? (fr - ((size_t)1 << 30)) / SB : 0);
        if (c->opt.adjoint_mem_limit)  // the limit covers these checkpoints and the segment buffers
            room = std::min(room, (long long)(c->opt.adjoint_mem_limit / SB) - nbuf);
        for (int k = 0; k < C; ++k) {
            void* p = nullptr;
            bool h = false;
            if (room > 0 && (p = dev_alloc(c, SB))) --room;
            if (!p) {
                if (cudaMallocHost(&p, SB) != cudaSuccess) {
                    (void)cudaGetLastError();
                    release();
                    return fail(c, LBM_ERR_OOM, "adjoint checkpoint %d (%zu bytes, host)", k, SB);
                }
                h = true;
            }
            ckpt[k] = p;
            ckpt_host[k] = h;
            own.push_back(p);
            own_host.push_back(h);
        }
        const int init_layout = c->scheme == LBM_PULL2 ? LAYOUT_PULL : LAYOUT_LOCAL;
        LBM_ADJ_CHECK(c->ops->init(c->geom, cf, init_layout, c->rho_init_null ? nullptr : c->rho_init,
                                   c->u_init_null ? nullptr : c->u_init, bufs[0], c->stream),
                      "adjoint init");
        c->launches += 1;
        int sb = 0;
        for (long long t = 0; t < n; ++t) {
            if (t % K == 0)
                LBM_ADJ_CHECK(cudaMemcpyAsync(ckpt[t / K], bufs[sb], SB, cudaMemcpyDefault, c->stream),
                              "checkpoint copy");
            LBM_ADJ_RC(step_oop(bufs[sb], bufs[sb ^ 1], t, "forward recompute"));
            sb ^= 1;
        }
    }

    // Host checkpoints are restored into bufs[0] (segments with even index) and one extra buffer
    // (odd index); with that buffer, the restore of segment s-1 runs on a copy stream while
    // segment s is recomputed and swept. Without room for it, restores are synchronous.
    void* rbuf[2] = {bufs[0], nullptr};
    int n_host = 0, n_dev = 0;
    for (int k = 0; k < C; ++k) (ckpt_host[k] ? n_host : n_dev) += 1;
    // the extra state must fit next to the device checkpoints and the segment plan
    bool room1 = (long long)c->adj_bufs.size() > nbuf;
    if (!room1) {
        LBM_ADJ_CHECK(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
        room1 = fr > SB + ((size_t)1 << 30);
    }
    if (c->opt.adjoint_mem_limit) room1 = room1 && (size_t)(n_dev + nbuf + 1) * SB <= c->opt.adjoint_mem_limit;
    if (n_host > 1 && room1) {
        if ((long long)c->adj_bufs.size() <= nbuf) {
            void* p = dev_alloc(c, SB);
            if (p) {
                c->adj_bufs.push_back(p);
                bufs = c->adj_bufs.data();
                rbuf[0] = bufs[0];
                LBM_ADJ_CHECK(cudaMemsetAsync(p, 0, SB, c->stream), "clear");
            }
        }
        if ((long long)c->adj_bufs.size() > nbuf) {
            rbuf[1] = bufs[nbuf];
            LBM_ADJ_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "copy stream");
            LBM_ADJ_CHECK(cudaEventCreateWithFlags(&ev_free, cudaEventDisableTiming), "event");
            LBM_ADJ_CHECK(cudaEventCreateWithFlags(&ev_done[0], cudaEventDisableTiming), "event");
            LBM_ADJ_CHECK(cudaEventCreateWithFlags(&ev_done[1], cudaEventDisableTiming), "event");
        }
    }
    std::vector<bool> issued(C, false);
    int prefetched = 0;
    // Restore of host checkpoint s on the copy stream, after all work enqueued so far on the
    // context's stream (the previous user of its buffer is the segment two places later).
    auto prefetch = [&](int s) -> cudaError_t {
        cudaError_t e = cudaEventRecord(ev_free, c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_free, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rbuf[s & 1], ckpt[s], SB, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_done[s & 1], cs);
        issued[s] = true;
        ++prefetched;
        return e;
    };

    // Seed from f(n), the context's current state.
    int lc = 0;
    LBM_ADJ_CHECK(c->ops->adj_seed(c->geom, cf, layout_now(c, n), state_ptr(c), loss_grad, c->lam[lc], c->stream),
                  "adjoint seed");
    c->launches += 1;
    LBM_ADJ_RC(run_halo(c, LBM_HALO_ADJOINT, c->lam[lc]));
    if (cs && ckpt_host[C - 1]) LBM_ADJ_CHECK(prefetch(C - 1), "checkpoint prefetch");
    // adjoint steps t1+len-1 .. t1 over states held in st[0..len-1]
    auto sweep = [&](const std::vector<const void*>& st, long long t1) -> int {
        for (int j = (int)st.size() - 1; j >= 0; --j) {
            const cudaError_t e = c->ops->adj_step(c->geom, cf, layout_now(c, t1 + j), st[j], c->lam[lc],
                                                   c->lam[lc ^ 1], c->gpart, c->stream);
            c->launches += 1;
            lc ^= 1;
            if (e != cudaSuccess) return cuda_fail(c, e, "adjoint step");
            if (int rc = run_halo(c, LBM_HALO_ADJOINT, c->lam[lc])) return rc;
        }
        return LBM_OK;
    };
    // Small boxes are launch-bound: a full segment of a flat plan (K - 1 recompute steps and K
    // adjoint steps over the same buffers) is captured once as a CUDA graph and replayed for
    // every full segment, its start state first copied into bufs[0]. That needs the same lambda
    // and AA parities at every segment start (K even), device checkpoints only (bufs[0] is then
    // not a restore target), and no halo callbacks between the kernels.
    int n_host_ckpt = 0;
    for (int k = 0; k < C; ++k) n_host_ckpt += ckpt_host[k] ? 1 : 0;
    const bool seg_graphs = flat_plan && K % 2 == 0 && K >= 2 && n_host_ckpt == 0 && !c->slab &&
                            (c->opt.use_graphs > 0 || (c->opt.use_graphs == 0 && c->N <= (1LL << 21)));
    auto capture_segment = [&](long long t0) -> int {
        if (!c->cap_stream) LBM_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        LBM_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int j = 1; j < K && e == cudaSuccess; ++j) e = step_kernel(c, bufs[j - 1], bufs[j], t0 + j - 1, c->cap_stream);
        int l = lc;
        for (int j = K - 1; j >= 0 && e == cudaSuccess; --j) {
            e = c->ops->adj_step(c->geom, cf, layout_now(c, t0 + j), bufs[j], c->lam[l], c->lam[l ^ 1], c->gpart,
                                 c->cap_stream);
            l ^= 1;
        }
        cudaGraph_t gr = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &gr);
        if (e != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            return cuda_fail(c, e, "kernel launch during segment capture");
        }
        if (ee != cudaSuccess) return cuda_fail(c, ee, "cudaStreamEndCapture (segment)");
        const cudaError_t ie = cudaGraphInstantiate(&seg_graph, gr, 0);
        cudaGraphDestroy(gr);
        if (ie != cudaSuccess) {
            seg_graph = nullptr;
            return cuda_fail(c, ie, "cudaGraphInstantiate (segment)");
        }
        return LBM_OK;
    };
    // Reverse sweep over segments.
    for (int s = C - 1; s >= 0; --s) {
        const long long t0 = (long long)s * K;
        const int len = (int)std::min<long long>(K, n - t0);
        const void* start = ckpt[s];
        if (ckpt_host[s]) {
            if (issued[s]) {
                LBM_ADJ_CHECK(cudaStreamWaitEvent(c->stream, ev_done[s & 1], 0), "checkpoint wait");
                start = rbuf[s & 1];
            } else {
                LBM_ADJ_CHECK(cudaMemcpyAsync(bufs[0], ckpt[s], SB, cudaMemcpyHostToDevice, c->stream),
                              "checkpoint restore");
                start = bufs[0];
            }
        }
        if (cs && s > 0 && ckpt_host[s - 1]) LBM_ADJ_CHECK(prefetch(s - 1), "checkpoint prefetch");
        if (seg_graphs && len == K) {
            if (start != bufs[0])
                LBM_ADJ_CHECK(cudaMemcpyAsync(bufs[0], start, SB, cudaMemcpyDeviceToDevice, c->stream),
                              "segment start copy");
            if (!seg_graph) LBM_ADJ_RC(capture_segment(t0));
            LBM_ADJ_CHECK(cudaGraphLaunch(seg_graph, c->stream), "segment graph launch");
            c->launches += 2 * K - 1;  // K even: lc is back at its value at the segment start
        } else {
            std::vector<int> sp;
            segment_plan(len, W, sp);  // W admits a plan for K >= len steps
            const int m = (int)sp.size() - 1;
            if (m == 0) {  // flat: states t0 + j in bufs[j], j = 1 .. len-1
                std::vector<const void*> st(len);
                st[0] = start;
                for (int j = 1; j < len; ++j) {
                    LBM_ADJ_RC(step_oop(st[j - 1], bufs[j], t0 + j - 1, "segment recompute"));
                    st[j] = bufs[j];
                }
                LBM_ADJ_RC(sweep(st, t0));
            } else {  // states s_1 .. s_(m-1) in bufs[1 .. m-1], the last sub-segment in bufs[m ..]
                void** last = bufs + m;
                const int L = len - sp[m];
                const void* cur = start;
                for (int i = 1, j = 1; i < len; ++i) {
                    void* dst;
                    if (j < m && i == sp[j])
                        dst = bufs[j++];
                    else if (i >= sp[m])
                        dst = last[i - sp[m]];
                    else  // not kept: alternate the last two buffers, state s_m - 1 in last[L - 1]
                        dst = last[L - 1 - ((sp[m] - 1 - i) & 1)];
                    LBM_ADJ_RC(step_oop(cur, dst, t0 + i - 1, "sub-checkpoint recompute"));
                    cur = dst;
                }
                std::vector<const void*> st(last, last + L);
                LBM_ADJ_RC(sweep(st, t0 + sp[m]));
                for (int j = m - 1; j >= 0; --j) {
                    const int lj = sp[j + 1] - sp[j];  // <= L + 1
                    st.assign(lj, nullptr);
                    st[0] = j == 0 ? start : bufs[j];
                    for (int i = 1; i < lj; ++i) {
                        LBM_ADJ_RC(step_oop(st[i - 1], last[i - 1], t0 + sp[j] + i - 1, "segment recompute"));
                        st[i] = last[i - 1];
                    }
                    LBM_ADJ_RC(sweep(st, t0 + sp[j]));
                }
            }
        }
    }
    // Through f(0) = feq(rho0, u0; Theta).
    LBM_ADJ_CHECK(c->ops->adj_init(c->geom, cf, c->rho_init_null ? nullptr : c->rho_init,
                                   c->u_init_null ? nullptr : c->u_init, c->lam[lc], c->du0, c->gpart, c->stream),
                  "adjoint init gradient");
    LBM_ADJ_CHECK(reduce_partials(c->gpart, c->shape.nblocks, 8, c->dout, c->stream), "gradient reduction");
    c->launches += 2;
    LBM_ADJ_CHECK(cudaMemcpyAsync(c->hout, c->dout, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                  "gradient copy");
    LBM_ADJ_CHECK(cudaStreamSynchronize(c->stream), "adjoint sync");
#undef LBM_ADJ_CHECK
#undef LBM_ADJ_RC
    if (c->d == 3) {
        for (int k = 0; k < 6; ++k) c->grad_theta[k] = c->hout[k];
    } else {
        c->grad_theta[0] = c->hout[0];
        c->grad_theta[1] = c->hout[1];
        c->grad_theta[2] = c->hout[3];
    }
    c->grad_tau = c->hout[6];
    c->grads_ready = true;
    c->last_adj_K2 = longest;
    c->last_adj_prefetch = prefetched;
    release();
    return LBM_OK;
}

int lbm_adjoint_info(const lbm_ctx* c, int* sub_segment, int* prefetched) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (sub_segment) *sub_segment = c->last_adj_K2;
    if (prefetched) *prefetched = c->last_adj_prefetch;
    return LBM_OK;
}

int lbm_adjoint_plan(int len, int working, int* starts, int capacity, int* count) {
    if (len < 1 || working < 0 || !starts || !count || capacity < 1) return LBM_ERR_INVALID_ARG;
    std::vector<int> sp;
    if (!segment_plan(len, working, sp)) return LBM_ERR_OOM;
    *count = (int)sp.size();
    if ((int)sp.size() > capacity) return LBM_ERR_INVALID_ARG;
    for (size_t j = 0; j < sp.size(); ++j) starts[j] = sp[j];
    return LBM_OK;
}

int lbm_adjoint_release(lbm_ctx* c) {
    if (!c) return LBM_ERR_INVALID_ARG;
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    const size_t SB = c->state_bytes(), LB = (size_t)c->q * c->N * c->felem;
    for (void* p : c->adj_bufs) dev_free(c, p, SB);
    c->adj_bufs.clear();
    dev_free(c, c->lam[0], LB);
    dev_free(c, c->lam[1], LB);
    c->lam[0] = c->lam[1] = nullptr;
    return LBM_OK;
}

int lbm_gradients(lbm_ctx* c, double* dTheta, double* dtau, void* du0) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (int rc = flow_only(c, "lbm_gradients")) return rc;
    if (!c->grads_ready) return fail(c, LBM_ERR_STATE, "lbm_gradients before a successful lbm_adjoint");
    if (dTheta)
        for (int k = 0; k < (c->d == 3 ? 6 : 3); ++k) dTheta[k] = c->grad_theta[k];
    if (dtau) *dtau = c->grad_tau;
    if (du0) {
        LBM_CUDA(c, cudaMemcpyAsync(du0, c->du0, (size_t)c->d * c->N * c->felem, cudaMemcpyDefault, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------------
// Save / resume
// ---------------------------------------------------------------------------------------------
struct lbm_state_header {
    char magic[8];
    int32_t version, lattice, nx, ny, nz, storage, scheme, order;
    int64_t steps;
    int64_t reserved[4];
};

int lbm_state_bytes(const lbm_ctx* c, size_t* bytes) {
    if (!c || !bytes) return LBM_ERR_INVALID_ARG;
    *bytes = sizeof(lbm_state_header) + c->state_bytes();
    return LBM_OK;
}

int lbm_get_state(lbm_ctx* c, void* dst, size_t bytes) {
    if (!c || !dst) return LBM_ERR_INVALID_ARG;
    if (!c->state_valid) return fail(c, LBM_ERR_STATE, "no state to save");
    if (bytes < sizeof(lbm_state_header) + c->state_bytes()) return fail(c, LBM_ERR_INVALID_ARG, "buffer too small");
    lbm_state_header h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "LBMSTAT", 8);
    h.version = 1;
    h.lattice = c->q;
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.storage = c->storage;
    h.scheme = c->scheme;
    h.order = c->order;
    h.steps = c->steps;
    h.reserved[0] = c->kind;
    LBM_CUDA(c, cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyDefault, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync((char*)dst + sizeof(h), state_ptr(c), c->state_bytes(), cudaMemcpyDefault,
                                c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_state(lbm_ctx* c, const void* src, size_t bytes) {
    if (!c || !src) return LBM_ERR_INVALID_ARG;
    if (bytes < sizeof(lbm_state_header) + c->state_bytes()) return fail(c, LBM_ERR_INVALID_ARG, "buffer too small");
    lbm_state_header h;
    LBM_CUDA(c, cudaMemcpy(&h, src, sizeof(h), cudaMemcpyDefault));
    if (std::memcmp(h.magic, "LBMSTAT", 8) != 0 || h.version != 1 || h.lattice != c->q || h.nx != c->nx ||
        h.ny != c->ny || h.nz != c->nz || h.storage != c->storage || h.scheme != c->scheme || h.reserved[0] != c->kind)
        return fail(c, LBM_ERR_INVALID_ARG, "state does not match this context");
    c->cur = 0;
    LBM_CUDA(c, cudaMemcpyAsync(c->pop[0], (const char*)src + sizeof(h), c->state_bytes(), cudaMemcpyDefault,
                                c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->steps = h.steps;
    c->state_valid = true;
    c->init_fields = false;  // the adjoint needs the initial fields of an lbm_init
    c->grads_ready = false;
    c->rec_valid = 0;
    return LBM_OK;
}

int lbm_steps_done(const lbm_ctx* c, long long* steps) {
    if (!c || !steps) return LBM_ERR_INVALID_ARG;
    *steps = c->steps;
    return LBM_OK;
}

int lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_ERR_INVALID_ARG;
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    LBM_CUDA(c, cudaGetLastError());
    return LBM_OK;
}

int lbm_device_bytes(const lbm_ctx* c, size_t* bytes) {
    if (!c || !bytes) return LBM_ERR_INVALID_ARG;
    *bytes = c->dev_bytes;
    return LBM_OK;
}

int lbm_launch_count(const lbm_ctx* c, long long* launches) {
    if (!c || !launches) return LBM_ERR_INVALID_ARG;
    *launches = c->launches;
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------------
// Z-slab halo planes
// ---------------------------------------------------------------------------------------------
int lbm_halo_bytes(const lbm_ctx* c, int kind, size_t* bytes) {
    if (!c || !bytes || !c->slab || (kind != LBM_HALO_POPULATIONS && kind != LBM_HALO_ADJOINT))
        return LBM_ERR_INVALID_ARG;
    *bytes = halo_bytes_of(c, kind);
    return LBM_OK;
}

static int halo_call(lbm_ctx* c, int kind, int side, bool pack, void* array, void* buf) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!c->slab) return fail(c, LBM_ERR_INVALID_ARG, "halo planes exist only in z-slab contexts");
    if ((kind != LBM_HALO_POPULATIONS && kind != LBM_HALO_ADJOINT) || (side != 0 && side != 1) || !array || !buf)
        return fail(c, LBM_ERR_INVALID_ARG, "halo %s: bad kind, side or pointer", pack ? "pack" : "unpack");
    const cudaError_t e = halo_copy(c, kind, side, pack, array, buf);
    if (e != cudaSuccess) return cuda_fail(c, e, pack ? "halo pack" : "halo unpack");
    return LBM_OK;
}

int lbm_halo_pack(lbm_ctx* c, int kind, int side, const void* array, void* buf) {
    return halo_call(c, kind, side, true, const_cast<void*>(array), buf);
}

int lbm_halo_unpack(lbm_ctx* c, int kind, int side, void* array, const void* buf) {
    return halo_call(c, kind, side, false, array, const_cast<void*>(buf));
}

// ---------------------------------------------------------------------------------------------
// Anisotropic advection-diffusion of a scalar (lbm_ade.cuh).
// ---------------------------------------------------------------------------------------------
int lbm_ade_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, double tau, const double* Theta,
                   const uint8_t* solid_mask, const lbm_options* opt) {
    if (opt && opt->z_halo) {  // z-slabs are built for the flow only
        if (out) *out = nullptr;
        return LBM_ERR_INVALID_ARG;
    }
    const int rc = lbm_create_ex(out, lattice, nx, ny, nz, tau, Theta, solid_mask, opt);
    if (rc == LBM_OK) {
        lbm_ctx* c = *out;
        c->kind = 1;
        if (c->scheme != LBM_PULL2) {  // the scalar's AA steps run over the grid: no fluid-cell list
            dev_free(c, c->cell_idx, (size_t)c->cells.count * 4 + 4);
            c->cell_idx = nullptr;
            c->cells = CellList{};
        }
    }
    return rc;
}

static int ade_field(lbm_ctx* c) {
    if (c->ade_u) return LBM_OK;
    const size_t bytes = (size_t)c->d * c->N * c->felem;
    c->ade_u = dev_alloc(c, bytes);
    if (!c->ade_u) return fail(c, LBM_ERR_OOM, "advecting-velocity field (%zu bytes)", bytes);
    LBM_CUDA(c, cudaMemsetAsync(c->ade_u, 0, bytes, c->stream));
    return LBM_OK;
}

static void ade_use_field(lbm_ctx* c, bool zero) {
    if (c->ade_u_zero != zero) drop_graph(c);  // a captured step holds the field pointer or null
    c->ade_u_zero = zero;
}

int lbm_ade_set_velocity(lbm_ctx* c, const void* u, const double* u_const) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (c->kind != 1) return fail(c, LBM_ERR_INVALID_ARG, "lbm_ade_set_velocity: not a scalar context");
    if (u && u_const) return fail(c, LBM_ERR_INVALID_ARG, "give either a velocity field or a constant, not both");
    if (!u && !u_const) {
        ade_use_field(c, true);
        return LBM_OK;
    }
    if (u_const)
        for (int a = 0; a < c->d; ++a)
            if (!std::isfinite(u_const[a])) return fail(c, LBM_ERR_INVALID_ARG, "non-finite velocity");
    if (int rc = ade_field(c)) return rc;
    const size_t plane = (size_t)c->N * c->felem;
    if (u) {
        LBM_CUDA(c, cudaMemcpyAsync(c->ade_u, u, plane * c->d, cudaMemcpyDefault, c->stream));
    } else {
        for (int a = 0; a < c->d; ++a) {
            char* p = (char*)c->ade_u + a * plane;
            if (c->storage == LBM_FP64)
                k_fill<double><<<4 * 152, 256, 0, c->stream>>>((double*)p, c->N, u_const[a]);
            else
                k_fill<float><<<4 * 152, 256, 0, c->stream>>>((float*)p, c->N, (float)u_const[a]);
            LBM_CUDA(c, cudaGetLastError());
            c->launches += 1;
        }
    }
    ade_use_field(c, false);
    return LBM_OK;
}

int lbm_ade_velocity(lbm_ctx* c, void** u) {
    if (!c || !u) return LBM_ERR_INVALID_ARG;
    *u = nullptr;
    if (c->kind != 1) return fail(c, LBM_ERR_INVALID_ARG, "lbm_ade_velocity: not a scalar context");
    const bool fresh = c->ade_u == nullptr;
    if (int rc = ade_field(c)) return rc;
    if (!fresh && c->ade_u_zero) LBM_CUDA(c, cudaMemsetAsync(c->ade_u, 0, (size_t)c->d * c->N * c->felem, c->stream));
    ade_use_field(c, false);
    *u = c->ade_u;
    return LBM_OK;
}

}  // extern "C"
