// solve.cu -- solution of the normal equations M theta = rhs (Eq. 18).
//
// The paper names no solver.  M = C^T C is symmetric positive semidefinite;
// we factor the Jacobi-scaled matrix A = D M D (D = diag(M)^-1/2) by Cholesky
// in the plan's compute type (FP32 for the mixed path, FP64 for the plain
// path), form W = L^-1 explicitly, and refine with FP64 residuals:
//     r = rhs - M x (FP64),  x += D W^T W D r,
// until ||r|| / ||rhs|| <= 1e-12.
//
// Everything runs in one cooperative (grid-synchronised) kernel with two
// blocks per SM (FP32; one in FP64), so the ~n/NB dependent block steps cost
// a grid barrier each instead of a kernel launch:
//   * Cholesky, right-looking with NB-wide panels, NB = 32 (the default) or
//     64 (per plan; fewer barriers and trailing passes, a longer chain per
//     step: faster when several systems share a launch).  One block applies
//     the last update to the next diagonal block itself, factors it right
//     away and inverts the factor in the same sweep (factor_inv: eight steps
//     of four columns per 32x32 block, exchanging through shared memory;
//     factor64 builds the 64x64 block from two of them).  Phase P then forms
//     the panel L_ik = A_ik L_kk^-T as 64xNB GEMM tiles; phase U applies
//     A_ij -= L_ik L_jk^T to the trailing lower triangle in 64x64 tiles, on
//     the CUDA cores or, in the FP32 variant that asks for it, on the tensor
//     cores (tcgen05, 3xTF32 split; see tile_gemm_tc).
//   * W = L^-1 is formed in the same sweep (block forward elimination applied
//     to the identity): W_kk = L_kk^-1 from the diagonal factorisation, phase
//     P sets W_k[:, 0:k0] = L_kk^-1 W_k[:, 0:k0] and phase U applies
//     W_i -= L_ik W_k below.
//   * refinement: residual GEMV in FP64 and two GEMVs with W.
// Every control decision after a barrier uses values written before it, so
// all blocks execute the same sequence of barriers.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace sfft {

// Cholesky panel width NB (template parameter of the kernel): 32 or 64
constexpr int kNBMax = 64;
constexpr int kDB = 32;         // sub-block of the diagonal block factored in one sweep
constexpr int kKC = 32;         // k chunk of a tile product staged at once
constexpr int kTile = 64;       // trailing-update and GEMM output tile
constexpr int kMaxIters = 12;   // refinement iterations
constexpr double kTol = 1e-12;  // ||r|| / ||rhs||
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 2;  // resident FP32 solve blocks per SM (more loads in flight); FP64 takes 1
constexpr int kSeg = 8;         // row segments of the W^T y product
constexpr int kWDepth32 = 16;   // FP32 loads in flight per lane in the products with W
constexpr int kMaxBatch = kMaxSolveBatch;  // systems solved together by one launch

template <typename T>
struct SolveArgs {
    int n;
    const double *M, *rhs;
    double *dsc, *x, *r, *stats;  // stats[0..3]
    T *A, *W, *z, *y, *wseg;
    int *flag;  // [0] status (0 running, 1 converged, <0 failure), [1] iterations
    double *xout;
    sfft_solve_info *info;
};

template <typename T>
struct TileSmem {
    T a[kTile][kKC + 1];  // a(i, p)
    T b[kKC][kTile + 1];  // b(p, j)
};

// four consecutive values of shared memory (16-byte aligned)
__device__ __forceinline__ void ld4(const float *p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&o)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}

// Operands of one 32-deep chunk of a 64x64 tile product, loaded into
// registers (kLdOps elements of each per thread): all loads of a chunk are
// in flight before the first store to shared memory.
constexpr int kLdOps = kTile * kKC / kThreads;
template <typename T>
struct TileOps {
    T ra[kLdOps], rb[kLdOps];
};

// chunk [kk, kk + kn) of the operands of tile_gemm (same a, b, bounds)
template <bool TB, typename T>
__device__ __forceinline__ void tile_load(TileOps<T> &o, const T *Ag, int lda, int arow0, int arows, const T *Bg,
                                          int ldb, int bcol0, int bcols, int kk, int kn) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < kLdOps; ++q) {
        const int e = tid + q * kThreads, i = e / kKC, p = e % kKC;
        o.ra[q] = (i < arows && p < kn) ? Ag[(size_t)(arow0 + i) * lda + kk + p] : (T)0;
    }
    if constexpr (TB) {
#pragma unroll
        for (int q = 0; q < kLdOps; ++q) {
            const int e = tid + q * kThreads, j = e / kKC, p = e % kKC;
            o.rb[q] = (j < bcols && p < kn) ? Bg[(size_t)(bcol0 + j) * ldb + kk + p] : (T)0;
        }
    } else {
#pragma unroll
        for (int q = 0; q < kLdOps; ++q) {
            const int e = tid + q * kThreads, p = e / kTile, j = e % kTile;
            o.rb[q] = (j < bcols && p < kn) ? Bg[(size_t)(kk + p) * ldb + bcol0 + j] : (T)0;
        }
    }
}

// acc += the product of one loaded chunk: stage it in shared memory
// (tile_stage), then each thread accumulates its 4x4 outputs (rows 4 tr + u,
// columns tc + 16 v) over the 32 values of k in order (tile_compute).
template <bool TB, typename T>
__device__ __forceinline__ void tile_stage(TileSmem<T> &sm, const TileOps<T> &o) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < kLdOps; ++q) {
        const int e = tid + q * kThreads;
        sm.a[e / kKC][e % kKC] = o.ra[q];
        if constexpr (TB)
            sm.b[e % kKC][e / kKC] = o.rb[q];
        else
            sm.b[e / kTile][e % kTile] = o.rb[q];
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void tile_compute(T (&acc)[4][4], const TileSmem<T> &sm) {
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;
#pragma unroll 8
    for (int p = 0; p < kKC; ++p) {
        T av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) av[u] = sm.a[tr * 4 + u][p];
#pragma unroll
        for (int v = 0; v < 4; ++v) bv[v] = sm.b[p][tc + 16 * v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
    }
    __syncthreads();
}

template <bool TB, typename T>
__device__ __forceinline__ void tile_mul(T (&acc)[4][4], TileSmem<T> &sm, const TileOps<T> &o) {
    tile_stage<TB>(sm, o);
    tile_compute(acc, sm);
}

// 64x64 tile:  acc(i, j) += sum_{k0 <= k < k1} a(i, k) b(k, j)
//   a(i, k) = Ag[(arow0 + i) * lda + k]
//   b(k, j) = transB ? Bg[(bcol0 + j) * ldb + k] : Bg[k * ldb + bcol0 + j]
// rows i >= arows and columns j >= bcols read as zero.  All loads of a
// 32-deep chunk are issued before the first store to shared memory, so that
// their latencies overlap.
template <typename T>
__device__ void tile_gemm(T (&acc)[4][4], TileSmem<T> &sm, const T *Ag, int lda, int arow0, int arows,
                          const T *Bg, int ldb, int bcol0, int bcols, bool transB, int k0, int k1) {
    for (int kk = k0; kk < k1; kk += kKC) {
        TileOps<T> o;
        if (transB) {
            tile_load<true>(o, Ag, lda, arow0, arows, Bg, ldb, bcol0, bcols, kk, min(kKC, k1 - kk));
            tile_mul<true>(acc, sm, o);
        } else {
            tile_load<false>(o, Ag, lda, arow0, arows, Bg, ldb, bcol0, bcols, kk, min(kKC, k1 - kk));
            tile_mul<false>(acc, sm, o);
        }
    }
}

// ---- the FP32 tile GEMM on the tensor cores (tcgen05, sm_100 family) --------
// The 64x64x32 tile products of the trailing update run as tcgen05.mma of
// kind::tf32 (M = N = 64, K = 8 per instruction) with the accumulator in
// tensor memory.  TF32 keeps 10 mantissa bits, too few for a factor that
// must seed the FP64 refinement at a Jacobi-scaled condition number near
// 3e6, so each operand is split as v = hi + lo with hi = tf32(v) and
// lo = tf32(v - hi) (both rounded to nearest) and the tile product is
// accumulated as hi*hi + hi*lo + lo*hi ("3xTF32"): the dropped lo*lo term and
// the rounding of lo are below 2^-21 of each product, close to FP32.
// Operands are staged through registers into shared memory in the canonical
// K-major layout without swizzle: core matrices of 8 rows x 16 bytes, the
// next core matrix along K at +128 bytes (leading byte offset), the next
// 8-row group at +1024 bytes (stride byte offset, 32 K values per row).  One
// elected thread issues the 12 MMAs of a tile and commits them to an
// mbarrier; the block waits on it (bounded by a clock limit), reads the
// accumulator back with tcgen05.ld and hands it to the caller in the
// register layout of tile_gemm, through a shared transpose.  In tensor
// memory an M = 64 accumulator holds row 16 q + l in lane 32 q + l (q < 4,
// l < 16) and column j in column j.
constexpr int kTcCols = 64;                    // tensor-memory columns per block
constexpr long long kTcWaitCycles = 2000000000LL;  // bounded wait on the MMA barrier (~1 s)

struct __align__(1024) TcSmem {
    float op[4][kTile * kKC];  // a_hi, a_lo, b_hi, b_lo in the canonical K-major layout
};

// block-wide tensor-core state: the mbarrier, the accumulator's tensor-memory
// address, the phase of the next completion, and a sticky failure
struct TcState {
    uint64_t *mbar;
    uint32_t tmem;
    uint32_t phase;
    bool dead;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// canonical K-major position (floats) of element (row i, k) in a 64 x 32 tile
__device__ __forceinline__ int tc_pos(int i, int k) { return (((i >> 3) * 8 + (k >> 2)) << 5) + ((i & 7) << 2) + (k & 3); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ float tf32_rn(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// wait for completion `phase` of the mbarrier, at most kTcWaitCycles
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t phase) {
    const long long t0 = clock64();
    uint32_t done = 0;
    while (!done) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(mbar)), "r"(phase));
        if (!done && clock64() - t0 > kTcWaitCycles) return false;
    }
    return true;
}

__device__ void tc_init(TcState &st, uint64_t *mbar, uint32_t *slot) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                     "n"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    st.mbar = mbar;
    st.tmem = *slot;
    st.phase = 0;
    st.dead = false;
}

__device__ void tc_release(TcState &st) {
    if (st.dead) tc_wait(st.mbar, st.phase);  // a commit still outstanding: one more bounded wait
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(st.tmem), "n"(kTcCols));
}

// tile_gemm on the tensor cores for one chunk of at most kKC values of k
// (k1 - k0 <= kKC), same operands and result layout.  Returns false if the
// MMAs did not complete within the wait limit (acc is then not valid).
__device__ bool tile_gemm_tc(float (&acc)[4][4], TcSmem &tc, TcState &st, const float *Ag, int lda, int arow0,
                             int arows, const float *Bg, int ldb, int bcol0, int bcols, bool transB, int k0, int k1) {
    constexpr int kLd = kLdOps;
    const int tid = threadIdx.x, tr = tid / 16, tc16 = tid % 16;
    const int kn = min(kKC, k1 - k0);
    // element e = tid + q * kThreads of a 64 x 32 operand is (row, k) with
    // the lane choosing (row mod 8, k mod 4) and the rest (row / 8, k / 4):
    // a warp then stores one whole core matrix (32 consecutive words, no
    // bank conflict) and reads 8 rows x 16 bytes (or 4 k-rows x 32 bytes)
    float ra[kLd], rb[kLd];
    int ri[kLd], rk[kLd];
#pragma unroll
    for (int q = 0; q < kLd; ++q) {
        const int e = tid + q * kThreads, l = e & 31, hi = e >> 5;
        ri[q] = (hi & 7) * 8 + (l >> 2);
        rk[q] = (hi >> 3) * 4 + (l & 3);
    }
#pragma unroll
    for (int q = 0; q < kLd; ++q) {
        const int i = ri[q], pp = rk[q];
        ra[q] = (i < arows && pp < kn) ? Ag[(size_t)(arow0 + i) * lda + k0 + pp] : 0.f;
        rb[q] = (i < bcols && pp < kn)
                    ? (transB ? Bg[(size_t)(bcol0 + i) * ldb + k0 + pp] : Bg[(size_t)(k0 + pp) * ldb + bcol0 + i])
                    : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kLd; ++q) {
        const int pos = tc_pos(ri[q], rk[q]);
        const float ah = tf32_rn(ra[q]);
        tc.op[0][pos] = ah;
        tc.op[1][pos] = tf32_rn(ra[q] - ah);
        const float bh = tf32_rn(rb[q]);
        tc.op[2][pos] = bh;
        tc.op[3][pos] = tf32_rn(rb[q] - bh);
    }
    // the generic-proxy stores must be visible to the tensor core's reads
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0 && !st.dead) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTile >> 3) << 17) |
                                   ((uint32_t)(kTile >> 4) << 24);
        const uint32_t a0 = smem_addr(tc.op[0]), a1 = smem_addr(tc.op[1]);
        const uint32_t b0 = smem_addr(tc.op[2]), b1 = smem_addr(tc.op[3]);
#pragma unroll
        for (int ks = 0; ks < kKC / 8; ++ks) {
            const uint32_t off = ks * 256;  // two core matrices along K per MMA
            tc_mma(st.tmem, tc_desc(a0 + off), tc_desc(b0 + off), idesc, ks > 0);
            tc_mma(st.tmem, tc_desc(a0 + off), tc_desc(b1 + off), idesc, 1);
            tc_mma(st.tmem, tc_desc(a1 + off), tc_desc(b0 + off), idesc, 1);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(st.mbar)));
    }
    bool ok = !st.dead;
    if (ok) {
        ok = tc_wait(st.mbar, st.phase);
        st.phase ^= 1u;
    }
    // every thread takes the same decision (a timeout is seen by all but is
    // not guaranteed to be simultaneous): agree before touching the result
    ok = __syncthreads_and(ok);
    if (!ok) {
        st.dead = true;
        return false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    // accumulator -> shared transpose (over the operand tiles, whose reads
    // are complete) -> this thread's 4x4 entries
    float *Cs = &tc.op[0][0];  // 64 x 65
    const int warp = tid >> 5, lane = tid & 31, q = warp & 3, h = warp >> 2;
    uint32_t v[32];
    const uint32_t taddr = st.tmem + ((uint32_t)(32 * q) << 16) + 32 * h;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (lane < 16) {
        float *row = Cs + (16 * q + lane) * (kTile + 1) + 32 * h;
#pragma unroll
        for (int c = 0; c < 32; ++c) row[c] = __uint_as_float(v[c]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = Cs[(tr * 4 + u) * (kTile + 1) + tc16 + 16 * w];
    __syncthreads();  // the shared tiles are refilled by the next call
    return true;
}

// Shared memory of the diagonal-block factorisation (aliases the GEMM tiles):
// four columns of S (by row) and four rows of Y (by column) per step,
// double-buffered by step parity.
template <typename T>
struct __align__(16) FactorSmem {
    T col[2][kDB][4];
    T row[2][kDB][4];
    T lp[kNBMax][kKC + 1];  // staged operands (panel rows of the last update; 32 x 32 products)
    T s1[kDB][kDB + 1];  // L21
    T s2[kDB][kDB + 1];  // L21 L11^-1
};

template <typename T>
union SolveSmem {
    TileSmem<T> tile;
    FactorSmem<T> fac;
    TcSmem tc;  // FP32 only (the tensor-core tile GEMM)
};

template <typename T>
__device__ __forceinline__ T pick4(const T (&v)[4], int q) {
    return q == 0 ? v[0] : (q == 1 ? v[1] : (q == 2 ? v[2] : v[3]));
}

// 1 / sqrt(d): the FP32 factor only seeds the FP64 refinement, so the
// hardware approximation serves; FP64 takes the correctly rounded path.
__device__ __forceinline__ float inv_sqrt(float d) { return rsqrtf(d); }
__device__ __forceinline__ double inv_sqrt(double d) { return 1.0 / sqrt(d); }

// The whole block factors the 32x32 block of A at (k0, k0) (nb <= 32 rows
// inside the matrix) and inverts its factor in the same sweep, four columns
// per step.  With kp >= 0 the block first applies the last update of that
// block itself, S = A_kk - L L^T with L = A[k0:k0+32, kp:kp+32] (the panel
// of a 32-wide step kp), in the operation order of the trailing-update
// tiles; with kp < 0 A_kk is already fully updated.  Then:
// every thread factors the 4x4 pivot block itself, forms the L entries of the
// rows it needs by forward substitution, and applies the rank-4 update to S
// and the matching block forward elimination to Y (L Y = I, so Y ends as
// L^-1).  Thread (t, u) = (tid / 8, tid % 8) keeps row t, columns u, u+8,
// u+16, u+24 of S and Y in registers; each step publishes the next four
// columns of S and rows of Y through shared memory (one barrier per step).
// Writes L_kk into A and L_kk^-1 into W (zeros above the diagonal) and flags
// a non-positive pivot.
template <typename T>
__device__ void factor_inv(const SolveArgs<T> &s, FactorSmem<T> &f, int k0, int nb, int kp) {
    const int tid = threadIdx.x;
    const int n = s.n;
    const int t = tid >> 3, u = tid & 7;
    T sv[4], yv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = u + 8 * q;
        T v = (T)0;
        if (t < nb && c <= t) v = s.A[(size_t)(k0 + t) * n + k0 + c];  // the lower triangle only
        else if (t == c) v = (T)1;  // identity beyond the matrix edge
        sv[q] = v;
        yv[q] = (t == c) ? (T)1 : (T)0;
    }
    if (kp >= 0) {
#pragma unroll
        for (int q = 0; q < kDB * kDB / kThreads; ++q) {
            const int e = tid + q * kThreads, r = e / kDB, p = e % kDB;
            f.lp[r][p] = r < nb ? s.A[(size_t)(k0 + r) * n + kp + p] : (T)0;
        }
        __syncthreads();
        T acc[4] = {};
#pragma unroll 8
        for (int p = 0; p < kDB; ++p) {
            const T a = f.lp[t][p];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += a * f.lp[u + 8 * q][p];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (t < nb && u + 8 * q <= t) sv[q] = sv[q] - acc[q];
    }
    if (u < 4) f.col[0][t][u] = sv[0];
    if (t < 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) f.row[0][u + 8 * q][t] = yv[q];
    }
    bool bad = false;
    T minpiv = (T)1e30;
    // unrolled: buffer indices, register picks and row tests become constants
    // (one system 0.941 -> 0.912 ms at n = 1735)
#pragma unroll
    for (int jb = 0; jb < kDB; jb += 4) {
        __syncthreads();  // columns jb..jb+3 of S and rows jb..jb+3 of Y are published
        const int b = (jb >> 2) & 1;
        T p0[4], p1[4], p2[4], p3[4], st[4], sc[4][4], yc[4][4];
        ld4(f.col[b][jb], p0);
        ld4(f.col[b][jb + 1], p1);
        ld4(f.col[b][jb + 2], p2);
        ld4(f.col[b][jb + 3], p3);
        ld4(f.col[b][t], st);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ld4(f.col[b][u + 8 * q], sc[q]);
            ld4(f.row[b][u + 8 * q], yc[q]);
        }
        // 4x4 Cholesky of the pivot block
        const T d0 = p0[0];
        const T i0 = inv_sqrt(d0 > (T)0 ? d0 : (T)1);
        const T l10 = p1[0] * i0, l20 = p2[0] * i0, l30 = p3[0] * i0;
        const T d1 = p1[1] - l10 * l10;
        const T i1 = inv_sqrt(d1 > (T)0 ? d1 : (T)1);
        const T l21 = (p2[1] - l20 * l10) * i1, l31 = (p3[1] - l30 * l10) * i1;
        const T d2 = p2[2] - l20 * l20 - l21 * l21;
        const T i2 = inv_sqrt(d2 > (T)0 ? d2 : (T)1);
        const T l32 = (p3[2] - l30 * l20 - l31 * l21) * i2;
        const T d3 = p3[3] - l30 * l30 - l31 * l31 - l32 * l32;
        const T i3 = inv_sqrt(d3 > (T)0 ? d3 : (T)1);
        const T dp[4] = {d0, d1, d2, d3};
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (!(dp[p] > (T)0)) bad = true;
            if (jb + p < nb && dp[p] < minpiv) minpiv = dp[p];
        }
        // L entries in columns jb..jb+3 of a row from its S entries there
        auto lrow = [&](const T (&r)[4], T (&l)[4]) {
            l[0] = r[0] * i0;
            l[1] = (r[1] - l[0] * l10) * i1;
            l[2] = (r[2] - l[0] * l20 - l[1] * l21) * i2;
            l[3] = (r[3] - l[0] * l30 - l[1] * l31 - l[2] * l32) * i3;
        };
        T lt[4];
        lrow(st, lt);  // row t of L (entries right of the diagonal are not used)
        if (u < 4 && t < nb && jb + u < nb)
            s.A[(size_t)(k0 + t) * n + k0 + jb + u] = (t >= jb + u) ? pick4(lt, u) : (T)0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = u + 8 * q;
            // rows jb..jb+3 of X = L^-1 in column c: block forward substitution
            T x[4];
            lrow(yc[q], x);
            if (t >= jb && t < jb + 4 && c <= t && t < nb && c < nb)
                s.W[(size_t)(k0 + t) * n + k0 + c] = pick4(x, t - jb);
            if (t > jb + 3) {
                if (c > jb + 3 && c <= t) {
                    T lc[4];
                    lrow(sc[q], lc);
                    sv[q] -= lt[0] * lc[0] + lt[1] * lc[1] + lt[2] * lc[2] + lt[3] * lc[3];
                }
                if (c <= jb + 3) yv[q] -= lt[0] * x[0] + lt[1] * x[1] + lt[2] * x[2] + lt[3] * x[3];
            }
        }
        // publish columns jn..jn+3 of S and rows jn..jn+3 of Y (the other buffer)
        const int jn = jb + 4;
        if (jn < kDB) {
            const int u0 = jn & 7;
            if (u >= u0 && u < u0 + 4) f.col[b ^ 1][t][u - u0] = pick4(sv, jn >> 3);
            if (t >= jn && t < jn + 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) f.row[b ^ 1][u + 8 * q][t - jn] = yv[q];
            }
        }
    }
    // zeros above the diagonal of both blocks
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = u + 8 * q;
        if (c > t && t < nb && c < nb) {
            s.A[(size_t)(k0 + t) * n + k0 + c] = (T)0;
            s.W[(size_t)(k0 + t) * n + k0 + c] = (T)0;
        }
    }
    if (tid == 0) {
        if (bad) s.flag[0] = SFFT_ERR_SINGULAR;
        else if ((double)minpiv < s.stats[0]) s.stats[0] = (double)minpiv;
    }
    __syncthreads();
}

// 32x32 block product in the thread layout of factor_inv (thread (t, u)
// holds row t, columns u + 8 q): out(t, c) = sum_{p < 32} a(t, p) b(p, c),
// a at f.lp[0..31][p], b at f.lp[32 + p][c], accumulated over p in order.
template <typename T>
__device__ __forceinline__ void mm32(const FactorSmem<T> &f, T (&out)[4]) {
    const int tid = threadIdx.x, t = tid >> 3, u = tid & 7;
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = (T)0;
#pragma unroll 8
    for (int p = 0; p < kDB; ++p) {
        const T a = f.lp[t][p];
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] += a * f.lp[kDB + p][u + 8 * q];
    }
}

// The 64x64 diagonal block kb: with kp >= 0 the block first applies its last
// update A_kk -= L L^T, L = A[k0:k0+64, kp:kp+64] (the panel of step kp, two
// chunks of 32 in order, as the trailing-update tiles), to its lower
// triangle.  Then, with [L11 0; L21 L22] its factor,
//   L11 (factor_inv), L21 = A21 L11^-T, A22 -= L21 L21^T, L22 (factor_inv),
//   W21 = -L22^-1 (L21 L11^-1),
// so that W_kk = [L11^-1 0; W21 L22^-1] = L_kk^-1.  L_kk goes into A, L_kk^-1
// into W (zeros above the diagonal of both, over the whole 64x64 block).
template <typename T>
__device__ void factor64(const SolveArgs<T> &s, FactorSmem<T> &f, int kb, int kp) {
    constexpr int kNB = 64;
    const int tid = threadIdx.x, n = s.n;
    const int k0 = kb * kNB, nb = min(kNB, n - k0);
    if (kp >= 0) {
        const int tr = tid / 16, tc = tid % 16;  // rows 4 tr + a, columns tc + 16 v
        T acc[4][4] = {};
        for (int kc = 0; kc < kNB; kc += kKC) {
            for (int e = tid; e < kNB * kKC; e += kThreads) {
                const int r = e / kKC, p = e % kKC;
                f.lp[r][p] = r < nb ? s.A[(size_t)(k0 + r) * n + kp + kc + p] : (T)0;
            }
            __syncthreads();
#pragma unroll 8
            for (int p = 0; p < kKC; ++p) {
                T av[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) av[a] = f.lp[tr * 4 + a][p];
#pragma unroll
                for (int v = 0; v < 4; ++v) bv[v] = f.lp[tc + 16 * v][p];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[a][v] += av[a] * bv[v];
            }
            __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int r = tr * 4 + a, c = tc + 16 * v;
                if (r < nb && c <= r) {
                    T *p = s.A + (size_t)(k0 + r) * n + k0 + c;
                    *p = *p - acc[a][v];
                }
            }
        __syncthreads();  // the updated block is visible to the whole block
    }
    factor_inv(s, f, k0, min(kDB, nb), -1);
    const int n2 = nb - kDB;
    if (n2 <= 0) return;
    const int t = tid >> 3, u = tid & 7;
    T o[4];
    // L21 = A21 L11^-T: a(i, p) = A[k0+32+i][k0+p], b(p, c) = L11^-1[c][p]
    for (int e = tid; e < kDB * kDB; e += kThreads) {
        const int r = e / kDB, c = e % kDB;
        f.lp[r][c] = r < n2 ? s.A[(size_t)(k0 + kDB + r) * n + k0 + c] : (T)0;
        f.lp[kDB + r][c] = s.W[(size_t)(k0 + c) * n + k0 + r];
    }
    __syncthreads();
    mm32(f, o);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = u + 8 * q;
        f.s1[t][c] = t < n2 ? o[q] : (T)0;
        if (t < n2) s.A[(size_t)(k0 + kDB + t) * n + k0 + c] = o[q];
    }
    __syncthreads();
    // A22 -= L21 L21^T (lower triangle)
    for (int e = tid; e < kDB * kDB; e += kThreads) {
        const int r = e / kDB, c = e % kDB;
        f.lp[r][c] = f.s1[r][c];
        f.lp[kDB + r][c] = f.s1[c][r];
    }
    __syncthreads();
    mm32(f, o);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = u + 8 * q;
        if (t < n2 && c <= t) {
            T *p = s.A + (size_t)(k0 + kDB + t) * n + k0 + kDB + c;
            *p = *p - o[q];
        }
    }
    __syncthreads();
    factor_inv(s, f, k0 + kDB, n2, -1);
    // X = L21 L11^-1, then W21 = -L22^-1 X
    for (int e = tid; e < kDB * kDB; e += kThreads) {
        const int r = e / kDB, c = e % kDB;
        f.lp[r][c] = f.s1[r][c];
        f.lp[kDB + r][c] = s.W[(size_t)(k0 + r) * n + k0 + c];
    }
    __syncthreads();
    mm32(f, o);
#pragma unroll
    for (int q = 0; q < 4; ++q) f.s2[t][u + 8 * q] = o[q];
    __syncthreads();
    for (int e = tid; e < kDB * kDB; e += kThreads) {
        const int r = e / kDB, c = e % kDB;
        f.lp[r][c] = (r < n2 && c < n2) ? s.W[(size_t)(k0 + kDB + r) * n + k0 + kDB + c] : (T)0;
        f.lp[kDB + r][c] = f.s2[r][c];
    }
    __syncthreads();
    mm32(f, o);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = u + 8 * q;
        if (t < n2) s.W[(size_t)(k0 + kDB + t) * n + k0 + c] = -o[q];
        // above the diagonal: the upper-right quadrant of both blocks
        if (c < n2) {
            s.A[(size_t)(k0 + t) * n + k0 + kDB + c] = (T)0;
            s.W[(size_t)(k0 + t) * n + k0 + kDB + c] = (T)0;
        }
    }
    __syncthreads();
}

// diagonal block kb of an NB-wide factorisation, with the last update from
// the panel at column kp (kp < 0: none)
template <int NB, typename T>
__device__ __forceinline__ void factor_block(const SolveArgs<T> &s, FactorSmem<T> &f, int kb, int kp) {
    if constexpr (NB == kDB)
        factor_inv(s, f, kb * kDB, min(kDB, s.n - kb * kDB), kp);
    else
        factor64(s, f, kb, kp);
}

// pairwise sum of D partial sums (D a power of two) in a fixed order:
// neighbours first, ((a0 + a1) + (a2 + a3)) + ... 
template <typename T, int D>
__device__ __forceinline__ T tree_sum(T (&acc)[D]) {
#pragma unroll
    for (int s = 1; s < D; s *= 2)
#pragma unroll
        for (int q = 0; q + s < D; q += 2 * s) acc[q] = acc[q] + acc[q + s];
    return acc[0];
}

// sum_{j < len} a[j] b[j] by one warp (lane = this thread's lane), with
// D independent loads of each operand in flight; the result is reduced
// across the warp (every lane returns it).
template <typename T, typename V, int D = 8>
__device__ __forceinline__ T dot_warp(const T *a, const V *b, int lane, int len) {
    T acc[D];
#pragma unroll
    for (int q = 0; q < D; ++q) acc[q] = (T)0;
    int j = lane;
    for (; j + (D - 1) * 32 < len; j += D * 32) {
        T av[D], bv[D];
#pragma unroll
        for (int q = 0; q < D; ++q) {
            av[q] = a[j + 32 * q];
            bv[q] = (T)b[j + 32 * q];
        }
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] += av[q] * bv[q];
    }
    for (; j < len; j += 32) acc[0] += a[j] * (T)b[j];
    T r = tree_sum<T, D>(acc);
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

// sum_{k0 <= k < k1} W[k][i] y[k] by one thread, D rows in flight
template <typename T, int D = 8>
__device__ __forceinline__ T col_dot(const T *W, const T *y, int n, int i, int k0, int k1) {
    T acc[D];
#pragma unroll
    for (int q = 0; q < D; ++q) acc[q] = (T)0;
    int k = k0;
    for (; k + D - 1 < k1; k += D) {
        T wv[D], yv[D];
#pragma unroll
        for (int q = 0; q < D; ++q) {
            wv[q] = W[(size_t)(k + q) * n + i];
            yv[q] = y[k + q];
        }
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] += wv[q] * yv[q];
    }
    for (; k < k1; ++k) acc[0] += W[(size_t)k * n + i] * y[k];
    return tree_sum<T, D>(acc);
}

// loads in flight per lane in the refinement's products with W (compute type)
template <typename T>
__host__ __device__ constexpr int w_depth() { return sizeof(T) == 4 ? kWDepth32 : 8; }

// trailing-update tile tt -> (ti, tj), ti >= tj
__device__ __forceinline__ void lower_tile(int tt, int *ti, int *tj) {
    int t = tt, i = 0;
    while (t > i) {
        t -= i + 1;
        ++i;
    }
    *ti = i;
    *tj = t;
}

// Phase P task `task` of one system at panel k0: a 64-row tile of the panel
// L_ik = A_ik L_kk^-T (task < npt) or a 64-column tile of block row k of W,
// W_k[:, 0:k0] = L_kk^-1 W_k[:, 0:k0].  L_kk^-1 is held in W_kk.  Each tile
// reads its inputs into shared memory before it overwrites them.
template <typename T>
__device__ void panel_task(const SolveArgs<T> &s, TileSmem<T> &sm, int k0, int kn, int base, int npt, int task) {
    const int n = s.n, tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    const T *Linv = s.W + (size_t)k0 * n + k0;
    T acc[4][4] = {};
    if (task < npt) {
        const int i0 = base + task * kTile, ni = min(kTile, n - i0);
        // a(i, p) = A[i0 + i][k0 + p], b(p, c) = Linv[c][p]
        tile_gemm(acc, sm, s.A + k0, n, i0, ni, Linv, n, 0, kn, true, 0, kn);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int i = tr * 4 + u, j = tc + 16 * v;
                if (i < ni && j < kn) s.A[(size_t)(i0 + i) * n + k0 + j] = acc[u][v];
            }
    } else {
        const int j0 = (task - npt) * kTile, nj = min(kTile, k0 - j0);
        // a(r, p) = Linv[r][p], b(p, c) = W[k0 + p][j0 + c]
        tile_gemm(acc, sm, s.W + k0, n, k0, kn, s.W + (size_t)k0 * n, n, j0, nj, false, 0, kn);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int r = tr * 4 + u, c = tc + 16 * v;
                if (r < kn && c < nj) s.W[(size_t)(k0 + r) * n + j0 + c] = acc[u][v];
            }
    }
}

// Phase U task `task` of one system at panel k0 (panel width NB): a 64x64
// tile of the trailing lower triangle, A_ij -= L_ik L_jk^T (task < ntiles;
// task 0 holds the next diagonal block, whose last update factor_block
// applies itself: with NB = 32 that tile stores only its rows below it, with
// NB = 64 it is not a task), or a 64x64 tile of the block rows of W below,
// W_i[:, 0:k0+NB] -= L_ik W_k.  Columns k0..k0+NB-1 of W below the diagonal
// block are first written by this step, so their old values are zero and
// are not read (W is never cleared).  The products run over k in chunks of 32.
template <typename T>
struct UpdTile {
    int i0, j0, ni, nj;
    int rmin;       // first row stored
    bool wtile;     // a tile of W (else of A)
    TileOps<T> op;  // operands of the first chunk, loaded ahead of the product
};

template <int NB, typename T>
__device__ __forceinline__ void upd_desc(UpdTile<T> &u, const SolveArgs<T> &s, int k0, int base, int ntiles, int ncw,
                                         int task) {
    const int n = s.n;
    u.wtile = task >= ntiles;
    if (!u.wtile) {
        int ti, tj;
        lower_tile(task, &ti, &tj);
        u.i0 = base + ti * kTile;
        u.j0 = base + tj * kTile;
        u.nj = min(kTile, n - u.j0);
    } else {
        const int q = task - ntiles;
        u.i0 = base + (q / ncw) * kTile;
        u.j0 = (q % ncw) * kTile;
        u.nj = min(kTile, k0 + NB - u.j0);
    }
    u.ni = min(kTile, n - u.i0);
    u.rmin = (task == 0) ? base + NB : u.i0;
}

// a(i, p) = L[i0 + i][k0 + p]; b(p, j) = L[j0 + j][k0 + p] (A tile) or
// W[k0 + p][j0 + j] (W tile)
template <bool WT, typename T>
__device__ __forceinline__ void upd_load(UpdTile<T> &u, const SolveArgs<T> &s, int k0) {
    const int n = s.n;
    tile_load<!WT>(u.op, s.A + k0, n, u.i0, u.ni, WT ? s.W + (size_t)k0 * n : s.A + k0, n, u.j0, u.nj, 0, kKC);
}

// element (i, j) of the tile is stored (A: lower triangle; W: columns below k0 + NB)
template <bool WT, int NB>
__device__ __forceinline__ bool upd_in(int n, int k0, int rmin, int i, int j) {
    return i < n && i >= rmin && (WT ? j < k0 + NB : (j < n && j <= i));
}

template <bool WT, int NB, typename T>
__device__ __forceinline__ void upd_old(const UpdTile<T> &u, const SolveArgs<T> &s, int k0, T (&old)[4][4]) {
    const int n = s.n, tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    const T *C = WT ? s.W : s.A;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = u.i0 + tr * 4 + a, j = u.j0 + tc + 16 * v;
            old[a][v] = (upd_in<WT, NB>(n, k0, u.rmin, i, j) && !(WT && j >= k0)) ? C[(size_t)i * n + j] : (T)0;
        }
}

template <bool WT, int NB, typename T>
__device__ __forceinline__ void upd_store(const UpdTile<T> &u, const SolveArgs<T> &s, int k0, const T (&old)[4][4],
                                          const T (&acc)[4][4]) {
    const int n = s.n, tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    T *C = WT ? s.W : s.A;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = u.i0 + tr * 4 + a, j = u.j0 + tc + 16 * v;
            if (upd_in<WT, NB>(n, k0, u.rmin, i, j)) C[(size_t)i * n + j] = old[a][v] - acc[a][v];
        }
}

// the tile whose first operand chunk is in u.op: old values (their loads
// overlap the product), product on the CUDA cores (the loads of a later
// chunk are in flight during the product of the one before), store
template <bool WT, int NB, typename T>
__device__ __forceinline__ void upd_finish(const UpdTile<T> &u, const SolveArgs<T> &s, TileSmem<T> &sm, int k0) {
    T old[4][4], acc[4][4] = {};
    upd_old<WT, NB>(u, s, k0, old);
    tile_stage<!WT>(sm, u.op);
    const int n = s.n;
#pragma unroll
    for (int c = 1; c < NB / kKC; ++c) {
        TileOps<T> o;
        tile_load<!WT>(o, s.A + k0, n, u.i0, u.ni, WT ? s.W + (size_t)k0 * n : s.A + k0, n, u.j0, u.nj, c * kKC,
                       kKC);
        tile_compute(acc, sm);
        tile_stage<!WT>(sm, o);
    }
    tile_compute(acc, sm);
    upd_store<WT, NB>(u, s, k0, old, acc);
}

// One task on its own.  The tensor-core variant takes the tile product on
// the tensor cores in FP32 (3xTF32, per chunk of 32); a tensor-core wait that
// timed out flags the system (SFFT_ERR_TIMEOUT) and the tile is computed on
// the CUDA cores.
template <typename T, bool TC, int NB>
__device__ void update_task(const SolveArgs<T> &s, SolveSmem<T> &smu, TcState &st, int k0, int base, int ntiles,
                            int ncw, int task) {
    UpdTile<T> u;
    upd_desc<NB>(u, s, k0, base, ntiles, ncw, task);
    if constexpr (TC && sizeof(T) == 4) {
        const int n = s.n;
        T old[4][4], acc[4][4] = {};
        if (u.wtile)
            upd_old<true, NB>(u, s, k0, old);
        else
            upd_old<false, NB>(u, s, k0, old);
        const T *Bg = u.wtile ? s.W + (size_t)k0 * n : s.A + k0;
        bool ok = true;
        for (int kk = 0; kk < NB && ok; kk += kKC) {
            T part[4][4];
            ok = tile_gemm_tc(part, smu.tc, st, s.A + k0, n, u.i0, u.ni, Bg, n, u.j0, u.nj, !u.wtile, kk, kk + kKC);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[a][v] += part[a][v];
        }
        if (!ok) {
            if (threadIdx.x == 0) s.flag[0] = SFFT_ERR_TIMEOUT;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[a][v] = (T)0;
            tile_gemm(acc, smu.tile, s.A + k0, n, u.i0, u.ni, Bg, n, u.j0, u.nj, !u.wtile, 0, NB);
        }
        if (u.wtile)
            upd_store<true, NB>(u, s, k0, old, acc);
        else
            upd_store<false, NB>(u, s, k0, old, acc);
    } else if (u.wtile) {
        upd_load<true>(u, s, k0);
        upd_finish<true, NB>(u, s, smu.tile, k0);
    } else {
        upd_load<false>(u, s, k0);
        upd_finish<false, NB>(u, s, smu.tile, k0);
    }
}

// row i of A = D M D up to the diagonal, eight loads of each operand in flight per lane
template <typename T>
__device__ __forceinline__ void scale_row(const SolveArgs<T> &s, int i, int lane) {
    const int n = s.n;
    const double di = s.dsc[i];
    const double *Mi = s.M + (size_t)i * n;
    T *Ai = s.A + (size_t)i * n;
    for (int j0 = lane; j0 <= i; j0 += 8 * 32) {
        double m[8], d[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + 32 * q;
            m[q] = j <= i ? Mi[j] : 0.0;
            d[q] = j <= i ? s.dsc[j] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + 32 * q;
            if (j <= i) Ai[j] = (T)(m[q] * di * d[q]);
        }
    }
}

// Up to kMaxBatch systems, of equal or different sizes, solved together:
// every phase spreads the tasks of all systems over the grid, and block b
// factors the diagonal blocks of system b, so the serial chains of the
// systems run side by side.  Each system sees the operations of a solve on
// its own, in the same order.
template <typename T>
struct BatchArgs {
    int nsys;
    SolveArgs<T> sys[kMaxBatch];
};

// system of a flat task index, from the prefix sums offs[0..nsys]
__device__ __forceinline__ int sys_of(const int *offs, int nsys, int task) {
    int b = 0;
    while (b + 1 < nsys && task >= offs[b + 1]) ++b;
    return b;
}

template <typename T, bool TC, int NB>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kBlocksPerSM : 1) k_solve_coop(BatchArgs<T> ba) {
    cg::grid_group grid = cg::this_grid();
    __shared__ SolveSmem<T> sm;
    __shared__ double sums[kMaxBatch][2];
    __shared__ __align__(8) uint64_t tc_mbar;
    __shared__ uint32_t tc_slot;
    TcState st{};
    if constexpr (TC) tc_init(st, &tc_mbar, &tc_slot);
    const int tid = threadIdx.x, bid = blockIdx.x, nbk = gridDim.x;
    const int gtid = bid * kThreads + tid, gthreads = nbk * kThreads;
    const int warp = tid >> 5, lane = tid & 31, nw = kThreads / 32;
    const int nsys = ba.nsys;
    // sizes may differ between systems: rows of all systems as one flat range
    int nrow[kMaxBatch + 1];
    nrow[0] = 0;
    int nblk_max = 0;
    for (int b = 0; b < nsys; ++b) {
        nrow[b + 1] = nrow[b] + ba.sys[b].n;
        nblk_max = max(nblk_max, (ba.sys[b].n + NB - 1) / NB);
    }
    const int nrows_all = nrow[nsys];

    // ---- status reset; Jacobi scaling, zero W and x -------------------------
    if (bid == 0 && tid < nsys) {
        const SolveArgs<T> &s = ba.sys[tid];
        s.flag[0] = s.flag[1] = s.flag[2] = s.flag[3] = 0;
        s.stats[0] = 1e300;
        s.stats[1] = s.stats[2] = s.stats[3] = 0.0;
    }
    grid.sync();
    for (int b = 0; b < nsys; ++b) {
        const SolveArgs<T> &s = ba.sys[b];
        const int n = s.n;
        for (int i = gtid; i < n; i += gthreads) {
            const double d = s.M[(size_t)i * n + i];
            if (!(d > 0.0)) s.flag[0] = SFFT_ERR_SINGULAR;
            s.dsc[i] = (d > 0.0) ? 1.0 / sqrt(d) : 0.0;
            s.x[i] = 0.0;
        }
    }
    int wofs[kMaxBatch + 1];  // flat W^T y tasks of all systems
    int yofs[kMaxBatch + 1];  // flat row-pair tasks (k, n - 1 - k) of all systems
    wofs[0] = yofs[0] = 0;
    for (int b = 0; b < nsys; ++b) {
        wofs[b + 1] = wofs[b] + ((ba.sys[b].n + 31) / 32) * kSeg;
        yofs[b + 1] = yofs[b] + (ba.sys[b].n + 1) / 2;
    }
    grid.sync();
    // A = D M D on the lower triangle (nothing reads the upper one), one warp
    // per row pair (k, n - 1 - k)
    for (int task = bid * nw + warp; task < yofs[nsys]; task += nbk * nw) {
        const int b = sys_of(yofs, nsys, task), k = task - yofs[b];
        const SolveArgs<T> &s = ba.sys[b];
        scale_row(s, k, lane);
        if (s.n - 1 - k != k) scale_row(s, s.n - 1 - k, lane);
    }
    grid.sync();

    // ---- Cholesky and W = L^-1 ----------------------------------------------
    // A system whose status turned negative is skipped from then on, and one
    // whose panels are done waits for the larger ones.  The task counts must
    // be the same in every block, so each step reads the status flags once,
    // right after a barrier and before the update phase in which factor_inv
    // may write them again.
    if (bid < nsys && ba.sys[bid].flag[0] == 0) factor_block<NB>(ba.sys[bid], sm.fac, 0, -1);
    grid.sync();
    for (int kb = 0; kb < nblk_max; ++kb) {
        const int k0 = kb * NB;
        const int base = k0 + NB;  // first trailing row
        unsigned live = 0;
        for (int b = 0; b < nsys; ++b)
            if (kb < (ba.sys[b].n + NB - 1) / NB && ba.sys[b].flag[0] == 0) live |= 1u << b;
        int offs[kMaxBatch + 1];
        offs[0] = 0;
        for (int b = 0; b < nsys; ++b) {
            const SolveArgs<T> &s = ba.sys[b];
            int cnt = 0;
            if (live & (1u << b)) {
                const int rows = s.n - base;
                cnt = (rows > 0 ? (rows + kTile - 1) / kTile : 0) + (k0 + kTile - 1) / kTile;
            }
            offs[b + 1] = offs[b] + cnt;
        }
        for (int task = bid; task < offs[nsys]; task += nbk) {
            const int b = sys_of(offs, nsys, task);
            const SolveArgs<T> &s = ba.sys[b];
            const int rows = s.n - base;
            const int npt = rows > 0 ? (rows + kTile - 1) / kTile : 0;
            panel_task(s, sm.tile, k0, min(NB, s.n - k0), base, npt, task - offs[b]);
        }
        grid.sync();
        // Block b applies the last update to the next diagonal block of
        // system b (tile 0) and factors that block at once; the other blocks
        // share the remaining tiles of all systems.
        bool any = false;
        offs[0] = 0;
        for (int b = 0; b < nsys; ++b) {
            const SolveArgs<T> &s = ba.sys[b];
            const int rows = s.n - base;
            int per = 0;
            if ((live & (1u << b)) && rows > 0) {
                const int nt = (rows + kTile - 1) / kTile;
                // NB = 64: tile 0 is the diagonal block, not a task
                per = nt * (nt + 1) / 2 + nt * ((k0 + NB + kTile - 1) / kTile) - (NB == kTile ? 1 : 0);
                any = true;
            }
            offs[b + 1] = offs[b] + per;
        }
        if (!any) break;  // every system's panels are done (same in every block)
        if (bid < nsys) {
            const SolveArgs<T> &s = ba.sys[bid];
            const int rows = s.n - base;
            if ((live & (1u << bid)) && rows > 0) factor_block<NB>(s, sm.fac, kb + 1, k0);
        } else {
            for (int task = bid - nsys; task < offs[nsys]; task += nbk - nsys) {
                const int b = sys_of(offs, nsys, task);
                const SolveArgs<T> &s = ba.sys[b];
                const int nt = (s.n - base + kTile - 1) / kTile;
                update_task<T, TC, NB>(s, sm, st, k0, base, nt * (nt + 1) / 2, (k0 + NB + kTile - 1) / kTile,
                                       (NB == kTile ? 1 : 0) + task - offs[b]);
            }
        }
        grid.sync();
    }

    // ---- refinement ---------------------------------------------------------
    // done: bit b set once system b has converged, failed or run out of
    // iterations; every block derives it from the same values.  The norms
    // are sums over the rows in one fixed order (warp b of every block sums
    // system b), so the decisions do not depend on the grid or the batch.
    unsigned done = 0;
    for (int b = 0; b < nsys; ++b)
        if (ba.sys[b].flag[0] != 0) done |= 1u << b;
    const unsigned all = (1u << nsys) - 1u;
    if (warp < nsys) {
        const SolveArgs<T> &s = ba.sys[warp];
        const double bb = dot_warp<double>(s.rhs, s.rhs, lane, s.n);
        if (lane == 0) sums[warp][1] = bb;
    }
    __syncthreads();
    for (int it = 0; it <= kMaxIters && done != all; ++it) {
        // r = rhs - M x (FP64); z = D r
        for (int row = bid * nw + warp; row < nrows_all; row += nbk * nw) {
            const int b = sys_of(nrow, nsys, row), i = row - nrow[b];
            if (done & (1u << b)) continue;
            const SolveArgs<T> &s = ba.sys[b];
            const double a = dot_warp<double>(s.M + (size_t)i * s.n, s.x, lane, s.n);
            const double ri = s.rhs[i] - a;
            if (lane == 0) {
                s.r[i] = ri;
                s.z[i] = (T)(s.dsc[i] * ri);
            }
        }
        grid.sync();
        if (warp < nsys && !(done & (1u << warp))) {
            const SolveArgs<T> &s = ba.sys[warp];
            const double rr = dot_warp<double>(s.r, s.r, lane, s.n);
            if (lane == 0) sums[warp][0] = rr;
        }
        __syncthreads();
        for (int b = 0; b < nsys; ++b) {
            if (done & (1u << b)) continue;
            const SolveArgs<T> &s = ba.sys[b];
            const double rr = sums[b][0], bb = sums[b][1];
            const double rel = (bb > 0.0) ? sqrt(rr / bb) : sqrt(rr);
            if (bid == 0 && tid == 0) {
                s.stats[1] = bb;
                s.stats[2] = rr;
            }
            if (rel <= kTol || rr == 0.0) {
                if (bid == 0 && tid == 0) s.flag[0] = 1;
                done |= 1u << b;
            } else if (it == kMaxIters) {
                if (bid == 0 && tid == 0) s.flag[0] = SFFT_ERR_NOT_CONVERGED;
                done |= 1u << b;
            }
        }
        if (done == all) break;
        // y = W z  (W lower triangular; row i has i + 1 entries).  A warp task
        // takes rows k and n - 1 - k, n + 1 entries together, so that every
        // task has the same length.
        for (int task = bid * nw + warp; task < yofs[nsys]; task += nbk * nw) {
            const int b = sys_of(yofs, nsys, task), k = task - yofs[b];
            if (done & (1u << b)) continue;
            const SolveArgs<T> &s = ba.sys[b];
            const int i2 = s.n - 1 - k;
            const T a = dot_warp<T, T, w_depth<T>()>(s.W + (size_t)k * s.n, s.z, lane, k + 1);
            if (lane == 0) s.y[k] = a;
            if (i2 != k) {
                const T a2 = dot_warp<T, T, w_depth<T>()>(s.W + (size_t)i2 * s.n, s.z, lane, i2 + 1);
                if (lane == 0) s.y[i2] = a2;
            }
        }
        grid.sync();
        // w = W^T y in kSeg row segments (coalesced rows of W), summed in a fixed order
        for (int task = bid * nw + warp; task < wofs[nsys]; task += nbk * nw) {
            const int b = sys_of(wofs, nsys, task), q = task - wofs[b];
            if (done & (1u << b)) continue;
            const SolveArgs<T> &s = ba.sys[b];
            const int n = s.n;
            const int segrows = (n + kSeg - 1) / kSeg;
            const int ch = q / kSeg, sg = q % kSeg;
            const int i = ch * 32 + lane;
            const int k0 = max(ch * 32, sg * segrows), k1 = min(n, (sg + 1) * segrows);
            if (i < n) s.wseg[(size_t)sg * n + i] = col_dot<T, w_depth<T>()>(s.W, s.y, n, i, k0, k1);
        }
        grid.sync();
        for (int e = gtid; e < nrows_all; e += gthreads) {
            const int b = sys_of(nrow, nsys, e), i = e - nrow[b];
            if (done & (1u << b)) continue;
            const SolveArgs<T> &s = ba.sys[b];
            T a = (T)0;
#pragma unroll
            for (int sg = 0; sg < kSeg; ++sg) a += s.wseg[(size_t)sg * s.n + i];
            s.x[i] += s.dsc[i] * (double)a;
        }
        if (bid == 0 && tid < nsys && !(done & (1u << tid))) ba.sys[tid].flag[1] += 1;
        grid.sync();
    }
    // ---- results ------------------------------------------------------------
    for (int e = gtid; e < nrows_all; e += gthreads) {
        const int b = sys_of(nrow, nsys, e), i = e - nrow[b];
        ba.sys[b].xout[i] = ba.sys[b].x[i];
    }
    if (bid == 0 && tid < nsys) {
        const SolveArgs<T> &s = ba.sys[tid];
        if (s.info) {
            const int f = s.flag[0];
            s.info->status = (f == 1) ? SFFT_OK : (f == 0 ? SFFT_ERR_NOT_CONVERGED : f);
            s.info->iters = s.flag[1];
            s.info->rel_residual = (s.stats[1] > 0.0) ? sqrt(s.stats[2] / s.stats[1]) : sqrt(s.stats[2]);
            s.info->min_pivot = s.stats[0];
        }
    }
    if constexpr (TC) tc_release(st);
}

static size_t solve_dyn_smem(bool) { return 0; }

// Arguments of one system: the caller's M, rhs, x, info and the workspace.
template <typename T>
static SolveArgs<T> system_args(int n, const double *M, const double *rhs, double *x, sfft_solve_info *info,
                                double *dsc, double *xw, double *r, void *A, void *W, void *zv, int *flag) {
    SolveArgs<T> a;
    a.n = n;
    a.M = M;
    a.rhs = rhs;
    a.dsc = dsc;
    a.x = xw;
    a.r = r;
    a.stats = xw + n;
    a.A = (T *)A;
    a.W = (T *)W;
    a.z = (T *)zv;
    a.y = (T *)zv + n;
    a.wseg = (T *)zv + 2 * (size_t)n;
    a.flag = flag;
    a.xout = x;
    a.info = info;
    return a;
}

// the kernel variant: tile products on the tensor cores (FP32 only), panel
// width 32 or 64 (FP32 only; FP64 solves use 32)
static const void *solve_kernel(bool fp64, bool tc, int panel) {
    if (fp64) return (const void *)k_solve_coop<double, false, 32>;
    if (panel == 64) return tc ? (const void *)k_solve_coop<float, true, 64> : (const void *)k_solve_coop<float, false, 64>;
    return tc ? (const void *)k_solve_coop<float, true, 32> : (const void *)k_solve_coop<float, false, 32>;
}

template <typename T>
static cudaError_t launch_batch(const BatchArgs<T> &ba, int grid, cudaStream_t st, bool tc = false, int panel = 32) {
    if (grid <= ba.nsys) return cudaErrorInvalidConfiguration;  // blocks >= nsys take the shared tasks
    void *args[] = {(void *)&ba};
    const void *kern = solve_kernel(sizeof(T) == 8, tc, panel);
    return cudaLaunchCooperativeKernel(kern, grid, kThreads, args, solve_dyn_smem(sizeof(T) == 8), st);
}

template <typename T>
static cudaError_t solve_batch_t(Plan *const *plans, int count, const double *const *M, const double *const *rhs,
                                 double *const *x, sfft_solve_info *const *info, cudaStream_t st) {
    BatchArgs<T> ba;
    ba.nsys = count;
    for (int b = 0; b < count; ++b) {
        Plan *p = plans[b];
        ba.sys[b] = system_args<T>(p->n, M[b], rhs[b], x[b], info[b], p->dscale, p->xw, p->r, p->A, p->Wm, p->zv,
                                   p->flag);
    }
    // the tensor-core tile variant (tune_tc = 2, FP32 only) allocates tensor
    // memory, which limits it to one block per SM: its own grid
    const bool tc = sizeof(T) == 4 && plans[0]->tune_tc == 2 && plans[0]->solve_grid_tc > count;
    const int full = tc ? plans[0]->solve_grid_tc : plans[0]->solve_grid;
    const int sg = plans[0]->tune_sgrid;
    int grid = full;
    if (sg > count && sg <= full) {
        grid = sg;  // set by hand
    } else if (count == 1 && !tc && sizeof(T) == 4 && full >= 2 * kMaxSolveBatch) {
        // one system alone: one block per SM (the step's serial chain, not the
        // tile throughput, sets its time; 1.12 -> 1.02 ms at n = 1735); several:
        // every resident block (batches of 8 on 304 blocks measured 561 pairs/s
        // serving against 515 on 152)
        grid = full / kBlocksPerSM;
    }
    const cudaError_t err = launch_batch(ba, grid, st, tc, plans[0]->solve_panel);
    plans[0]->launches += 1;
    return err;
}

cudaError_t solve_batch(Plan *const *plans, int count, const double *const *M, const double *const *rhs,
                        double *const *x, sfft_solve_info *const *info, cudaStream_t s) {
    if (count < 1 || count > kMaxBatch) return cudaErrorInvalidValue;
    for (int b = 1; b < count; ++b)  // sizes may differ
        if (plans[b]->fp64 != plans[0]->fp64 || (!plans[0]->fp64 && plans[b]->solve_panel != plans[0]->solve_panel))
            return cudaErrorInvalidValue;
    return plans[0]->fp64 ? solve_batch_t<double>(plans, count, M, rhs, x, info, s)
                          : solve_batch_t<float>(plans, count, M, rhs, x, info, s);
}

cudaError_t solve_system(Plan *p, const double *M, const double *rhs, double *x, sfft_solve_info *info,
                         cudaStream_t s) {
    return solve_batch(&p, 1, &M, &rhs, &x, &info, s);
}

int solve_grid_size(bool fp64, bool tc) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t dsm = solve_dyn_smem(fp64);
    // all of the unified L1/shared storage as shared memory, so that two FP32
    // blocks (33 KB of static shared memory each) fit on an SM; the grid is
    // the smaller residency of the two panel widths
    per = 1 << 30;
    for (int panel = 32; panel <= (fp64 ? 32 : 64); panel += 32) {
        const void *kern = solve_kernel(fp64, tc, panel);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        int pk = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pk, kern, kThreads, dsm);
        per = pk < per ? pk : per;
    }
    if (per < 1 || sms < 1) return 0;
    const int g = sms * (per < kBlocksPerSM ? per : kBlocksPerSM);
    return g <= kMaxSolveGrid ? g : 0;
}

size_t solve_vec_elems(int n) { return (size_t)(2 + kSeg) * n; }

template <typename T>
static cudaError_t solve_buf_t(const SolveBuffers &b, const double *M, const double *rhs, double *x,
                               sfft_solve_info *info, cudaStream_t st) {
    BatchArgs<T> ba;
    ba.nsys = 1;
    ba.sys[0] = system_args<T>(b.n, M, rhs, x, info, b.dsc, b.xw, b.r, b.A, b.W, b.zv, b.flag);
    return launch_batch(ba, b.grid, st);
}

cudaError_t solve_on_buffers(const SolveBuffers &b, const double *M, const double *rhs, double *x,
                             sfft_solve_info *info, cudaStream_t s) {
    return b.fp64 ? solve_buf_t<double>(b, M, rhs, x, info, s) : solve_buf_t<float>(b, M, rhs, x, info, s);
}

}  // namespace sfft
