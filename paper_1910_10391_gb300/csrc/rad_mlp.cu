// Surrogate MLP for per-particle spectra: training and inference kernels.
//
// Network: x (n_in, FP32) -> [Linear -> GELU] x depth (width) -> Linear -> y (n_out, FP32).
// The first layer (the input features, n_in <= 64) runs in FP32 so inputs are not quantized;
// every other layer is a BF16 x BF16 -> FP32 GEMM on the fifth-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory) with the bias, GELU (exact erf form) and their
// derivatives fused into the GEMM epilogues. FP32 master weights are updated by AdamW
// (Loshchilov & Hutter, "Decoupled weight decay regularization", ICLR 2019) and copied to BF16
// for the GEMMs. Loss: mean squared error.
#include <cuda_bf16.h>
#include <math.h>

#include <atomic>
#include <cstdio>
#include <random>
#include <vector>

#include "rad_internal.cuh"

namespace rad {
namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

// ---- tcgen05 (fifth-generation tensor core) GEMM ----
// C[M x N] = sum_k A(m, k) B(k, n), BF16 operands, FP32 accumulation in tensor memory, epilogue
// epi(m, n, value, epi.aux(m, n)):
//   A(m, k) = A_KM ? A[m * lda + k] : A[k * lda + m]
//   B(k, n) = B_KN ? B[n * ldb + k] : B[k * ldb + n]
// Block tile 128 x 128, K in steps of 64, 128 threads. The threads stage both operand tiles in
// shared memory in the layouts without swizzle that the MMA reads through its matrix descriptors:
// core matrices of 8 x 8 elements in 128 bytes (K-major: 8 rows of 8 K; MN-major: 8 K of 8 rows,
// whichever way the source is contiguous), the two K groups of a 16-K slice 128 bytes apart,
// successive 8-row groups 256 bytes apart, one 4 KB slab per 16 K. One thread
// issues four tcgen05.mma (M = 128, N = 128, K = 16) per K step and commits them to the stage's
// mbarrier; with two stages the staging of one K step overlaps the MMAs of the previous one. The
// 128 x 128 FP32 accumulator occupies 128 tensor-memory columns; each warp reads its 32 lanes
// (rows) back with tcgen05.ld into shared memory (the stages are free by then), and the block
// passes the tile to the epilogue row by row, consecutive threads on consecutive columns, so the
// epilogue's global stores are coalesced. Block z covers the K range
// [z k_chunk, min(K, (z + 1) k_chunk)) (split K; k_chunk a multiple of 64). Every mbarrier wait is
// bounded: when one runs out the block records RAD_ETIMEOUT, waits (bounded) for the MMAs it
// issued, frees its tensor memory and skips the epilogue.
constexpr int kTcM = 128, kTcN = 128, kTcK = 64;
constexpr int kTcSlab = 4096;               // one 16-K slice of a 128-row operand tile
constexpr int kTcOperand = 4 * kTcSlab;     // 128 rows x 64 K
constexpr int kTcStage = 2 * kTcOperand;    // A and B tiles
constexpr int kTcTile = kTcM * (kTcN + 1) * 4;  // the accumulator tile for the epilogue, rows padded
constexpr int kTcData = 2 * kTcStage > kTcTile ? 2 * kTcStage : kTcTile;
constexpr int kTcSmem = kTcData + 32;       // stages / tile, two mbarriers, the tensor-memory address
constexpr uint32_t kTcCols = 128;           // tensor-memory columns: the FP32 accumulator

// byte offset of (row r, k) in an operand tile
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return static_cast<uint32_t>((k >> 4) * kTcSlab + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading-dimension byte offset (between the two
// K groups of 8, 128 B) and stride byte offset (between groups of 8 rows, 256 B), each in 16-byte
// units; descriptor version 1 (bits 46-47); no swizzle (layout type 0 in bits 61-63). The same
// offsets serve the K-major and the MN-major tiles.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(128 >> 4) << 16) |
         (static_cast<uint64_t>(256 >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9,
// 10-12 = 1), A and B K-major (bit 15, 16 = 0) or MN-major (1), N >> 3 in bits 17-22, M >> 4 in
// bits 24-28
template <bool A_KM, bool B_KN>
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((A_KM ? 0u : 1u) << 15) | ((B_KN ? 0u : 1u) << 16) |
         (static_cast<uint32_t>(kTcN >> 3) << 17) | (static_cast<uint32_t>(kTcM >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 lanes: lane l gets row (lane base + l)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One operand tile: rows [r0, r0 + 128) (below `rows`) x K [k0, k0 + 64) (below k_end), zero
// outside, as 1024 chunks of 8 consecutive elements of the source, 8 per thread. tc_load reads a
// thread's 8 chunks into registers (all loads in flight together), tc_store writes them to the
// tile. A K-major source (KM: K contiguous) is staged K-major: a chunk is 8 K of one row, and a
// warp reads 8 rows x 4 chunks (64 contiguous bytes of each row). A source with the rows
// contiguous is staged MN-major (the descriptor's major bit set): a chunk is 8 rows of one K, a
// core matrix holds 8 K x 8 rows, each K's 8 rows in 16 bytes, and a warp reads 8 K x 4 chunks
// (64 contiguous bytes of each K). Either way a quarter warp stores 128 contiguous bytes.
template <bool KM>
__device__ __forceinline__ void tc_chunk(int c, int &r, int &k) {
  if (KM) {  // r: the row, k: the first of 8 K
    r = ((c >> 6) << 3) | (c & 7);
    k = ((c >> 3) & 7) << 3;
  } else {   // r: the first of 8 rows, k: the K
    k = ((c >> 7) << 3) | (c & 7);
    r = ((c >> 3) & 15) << 3;
  }
}

// byte offset of a chunk in an MN-major tile: (8 rows from r, K k)
__device__ __forceinline__ uint32_t tc_off_mn(int r, int k) {
  return static_cast<uint32_t>((k >> 4) * kTcSlab + ((k >> 3) & 1) * 128 + (r >> 3) * 256 + (k & 7) * 16);
}

template <bool KM>
__device__ __forceinline__ void tc_load(uint4 (&v)[8], const bf16 *__restrict__ P, int ld, int r0, int rows, int k0,
                                        int k_end, bool vec, int tid) {
  const unsigned short *Q = reinterpret_cast<const unsigned short *>(P);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int r, kc;
    tc_chunk<KM>(tid + 128 * i, r, kc);
    const int row = r0 + r, k = k0 + kc;
    v[i] = make_uint4(0u, 0u, 0u, 0u);
    if (KM) {
      if (row < rows && k < k_end) {
        if (vec && k + 8 <= k_end) {
          v[i] = __ldg(reinterpret_cast<const uint4 *>(Q + static_cast<int64_t>(row) * ld + k));
        } else {
          uint32_t e[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) e[j] = k + j < k_end ? Q[static_cast<int64_t>(row) * ld + k + j] : 0u;
          v[i] = make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16), e[4] | (e[5] << 16), e[6] | (e[7] << 16));
        }
      }
    } else {
      if (k < k_end && row < rows) {
        if (vec && row + 8 <= rows) {
          v[i] = __ldg(reinterpret_cast<const uint4 *>(Q + static_cast<int64_t>(k) * ld + row));
        } else {
          uint32_t e[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) e[j] = row + j < rows ? Q[static_cast<int64_t>(k) * ld + row + j] : 0u;
          v[i] = make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16), e[4] | (e[5] << 16), e[6] | (e[7] << 16));
        }
      }
    }
  }
}

template <bool KM>
__device__ __forceinline__ void tc_store(unsigned char *dst, const uint4 (&v)[8], int tid) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int r, k;
    tc_chunk<KM>(tid + 128 * i, r, k);
    *reinterpret_cast<uint4 *>(dst + (KM ? tc_off(r, k) : tc_off_mn(r, k))) = v[i];
  }
}

template <bool A_KM, bool B_KN, class Epi>
__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, const bf16 *__restrict__ A, int lda,
                                                 const bf16 *__restrict__ B, int ldb, Epi epi, int k_chunk,
                                                 int *status) {
  extern __shared__ __align__(128) unsigned char tc_sm[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(tc_sm + kTcData);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(tc_sm + kTcData + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * kTcN;
  const int k_begin = blockIdx.z * k_chunk;
  const int k_end = min(K, k_begin + k_chunk);
  const int nkt = k_end > k_begin ? (k_end - k_begin + kTcK - 1) / kTcK : 0;
  if (warp == 0) {  // the whole warp allocates; the address lands in shared memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const bool a_vec = (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda & 7) == 0;
  const bool b_vec = (reinterpret_cast<uintptr_t>(B) & 15) == 0 && (ldb & 7) == 0;
  bool failed = false;
  int issued = 0;  // K steps whose MMAs were issued and committed
  // K step kt's operands are read into registers during step kt - 1 (while its MMAs run) and
  // stored once the MMAs of step kt - 2 have released the stage
  uint4 ra[8], rb[8];
  if (nkt > 0) {
    tc_load<A_KM>(ra, A, lda, m0, M, k_begin, k_end, a_vec, tid);
    tc_load<B_KN>(rb, B, ldb, n0, N, k_begin, k_end, b_vec, tid);
  }
  for (int kt = 0; kt < nkt; ++kt) {
    const int st = kt & 1;
    unsigned char *sa = tc_sm + st * kTcStage;
    unsigned char *sb = sa + kTcOperand;
    // the MMAs of K step kt - 2 read this stage: their commit is phase (kt - 2) / 2 of its barrier
    const bool ok = kt < 2 || mbar_wait_bounded(&bar[st], static_cast<uint32_t>((kt - 2) >> 1) & 1u);
    if (ok) {
      tc_store<A_KM>(sa, ra, tid);
      tc_store<B_KN>(sb, rb, tid);
    }
    fence_proxy_async();  // the staged tiles become visible to the tensor core's (async) proxy
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc_mma(tmem, tc_desc(a0 + ks * kTcSlab), tc_desc(b0 + ks * kTcSlab), tc_idesc<A_KM, B_KN>(),
               (kt | ks) != 0 ? 1u : 0u);
      tc_commit(&bar[st]);
    }
    issued = kt + 1;
    if (kt + 1 < nkt) {
      const int k1 = k_begin + (kt + 1) * kTcK;
      tc_load<A_KM>(ra, A, lda, m0, M, k1, k_end, a_vec, tid);
      tc_load<B_KN>(rb, B, ldb, n0, N, k1, k_end, b_vec, tid);
    }
  }
  // the last commit completes after every MMA issued before it
  bool done = true;
  if (issued > 0) done = mbar_wait_bounded(&bar[(issued - 1) & 1], static_cast<uint32_t>((issued - 1) >> 1) & 1u);
  if (__syncthreads_or(!done)) failed = true;
  if (failed) {
    if (tid == 0) set_status(status, RAD_ETIMEOUT);
  } else {
    tc_fence_after();
    float *tile = reinterpret_cast<float *>(tc_sm);  // [128][129]: row r at r * 129 (bank r + column)
    const int r = warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kTcN; c0 += 16) {
      uint32_t v[16];
      if (nkt > 0) {
        tc_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c0), v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) tile[r * (kTcN + 1) + c0 + j] = __uint_as_float(v[j]);
    }
    __syncthreads();
#pragma unroll 1
    for (int e0 = tid; e0 < kTcM * kTcN; e0 += 128 * 16) {
      float a[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = e0 + 128 * u, rr = e >> 7, cc = e & (kTcN - 1);
        a[u] = (m0 + rr < M && n0 + cc < N) ? epi.aux(m0 + rr, n0 + cc) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = e0 + 128 * u, rr = e >> 7, cc = e & (kTcN - 1);
        if (m0 + rr < M && n0 + cc < N) epi(m0 + rr, n0 + cc, tile[rr * (kTcN + 1) + cc], a[u]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// ---- epilogues ----
// epi.aux(m, n) loads what the epilogue of element (m, n) reads besides the accumulator (a
// block loads a batch of them before it stores any), epi(m, n, v, aux) stores.
struct EpiHidden {  // Z = acc + b; H = bf16(gelu(Z)); Z kept for the backward pass (may be null)
  const float *bias;
  float *Z;
  bf16 *H;
  int ld;
  __device__ float aux(int, int n) const { return __ldg(bias + n); }
  __device__ void operator()(int m, int n, float v, float b) const {
    const float z = v + b;
    const int64_t e = static_cast<int64_t>(m) * ld + n;
    if (Z) Z[e] = z;
    H[e] = __float2bfloat16(gelu(z));
  }
};
struct EpiOut {  // Y = acc + b (FP32)
  const float *bias;
  float *Y;
  int ld;
  __device__ float aux(int, int n) const { return __ldg(bias + n); }
  __device__ void operator()(int m, int n, float v, float b) const { Y[static_cast<int64_t>(m) * ld + n] = v + b; }
};
struct EpiGradAct {  // dZ = bf16(acc * gelu'(Z))
  const float *Z;
  bf16 *dZ;
  int ld;
  __device__ float aux(int m, int n) const { return __ldg(Z + static_cast<int64_t>(m) * ld + n); }
  __device__ void operator()(int m, int n, float v, float z) const {
    dZ[static_cast<int64_t>(m) * ld + n] = __float2bfloat16(v * gelu_grad(z));
  }
};
struct EpiStore {  // plain FP32 store
  float *C;
  int ld;
  __device__ float aux(int, int) const { return 0.f; }
  __device__ void operator()(int m, int n, float v, float) const { C[static_cast<int64_t>(m) * ld + n] = v; }
};

struct EpiPartial {  // split K: FP32 partial sums of K range z at ws[z][m][n]
  float *ws;
  int64_t mn;
  int ld;
  __device__ float aux(int, int) const { return 0.f; }
  __device__ void operator()(int m, int n, float v, float) const {
    ws[blockIdx.z * mn + static_cast<int64_t>(m) * ld + n] = v;
  }
};

// Sum of the split-K partials in a fixed order, then the GEMM's own epilogue.
template <class Epi>
__global__ void k_splitk_reduce(int M, int N, int S, const float *__restrict__ ws, Epi epi) {
  const int64_t mn = static_cast<int64_t>(M) * N;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < mn;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float v = 0.f;
    for (int z = 0; z < S; ++z) v += ws[z * mn + e];
    const int m = static_cast<int>(e / N), n = static_cast<int>(e % N);
    epi(m, n, v, epi.aux(m, n));
  }
}

// Split-K workspace: a grid of fewer than kSplitTarget blocks with K of 256 or more is split in K
// (at least two K steps of 64 per split) until about that many blocks run; then
// S x M x N <= 2 kSplitTarget x 128 x 128 floats.
constexpr int kSplitTarget = 2 * 152;
constexpr int64_t kSplitWsFloats = 2ll * kSplitTarget * kTcM * kTcN;

template <bool A_KM, bool B_KN, class Epi>
cudaError_t launch_gemm_tc(dim3 grid, int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb, Epi epi,
                           int k_chunk, int *status, cudaStream_t st) {
  // the dynamic shared memory above 48 KB, allowed once per instantiation and device
  static std::atomic<unsigned long long> allowed{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (!(allowed.load() & bit)) {
    e = cudaFuncSetAttribute(k_gemm_tc<A_KM, B_KN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    allowed.fetch_or(bit);
  }
  k_gemm_tc<A_KM, B_KN, Epi><<<grid, 128, kTcSmem, st>>>(M, N, K, A, lda, B, ldb, epi, k_chunk, status);
  return cudaGetLastError();
}

template <bool A_KM, bool B_KN, class Epi>
cudaError_t gemm(int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb, Epi epi, float *ws,
                 cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  cudaError_t e;
  int *status = device_status_word(&e);
  if (!status) return e;
  const int gx = (N + kTcN - 1) / kTcN, gy = (M + kTcM - 1) / kTcM;
  const int blocks = gx * gy;
  const int kt = (K + kTcK - 1) / kTcK;
  int S = 1;
  if (ws && blocks < kSplitTarget && kt >= 4) S = std::min(kt / 2, (kSplitTarget + blocks - 1) / blocks);
  const int64_t mn = static_cast<int64_t>(M) * N;
  while (S > 1 && S * mn > kSplitWsFloats) --S;
  const int k_chunk = ((kt + S - 1) / S) * kTcK;
  S = (K + k_chunk - 1) / k_chunk;
  if (S <= 1) return launch_gemm_tc<A_KM, B_KN, Epi>(dim3(gx, gy, 1), M, N, K, A, lda, B, ldb, epi, kt * kTcK, status, st);
  EpiPartial part{ws, mn, N};
  e = launch_gemm_tc<A_KM, B_KN, EpiPartial>(dim3(gx, gy, S), M, N, K, A, lda, B, ldb, part, k_chunk, status, st);
  if (e != cudaSuccess) return e;
  k_splitk_reduce<Epi><<<static_cast<unsigned>(std::min<int64_t>((mn + 255) / 256, 4096)), 256, 0, st>>>(
      M, N, S, ws, epi);
  return cudaGetLastError();
}

// First layer in FP32: Z1[b][n] = sum_k x[b][k] W1[n][k] + b1[n]; H1 = bf16(gelu(Z1)).
__global__ void k_layer1(int64_t B, int n_in, int width, const float *__restrict__ x, const float *__restrict__ W,
                         const float *__restrict__ bias, float *Z, bf16 *H) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= B * width) return;
  const int64_t b = e / width;
  const int n = static_cast<int>(e % width);
  float z = bias[n];
  for (int k = 0; k < n_in; ++k) z = fmaf(x[b * n_in + k], W[n * n_in + k], z);
  if (Z) Z[e] = z;
  H[e] = __float2bfloat16(gelu(z));
}

// First-layer weight gradient in FP32: dW1[n][k] = sum_b dZ1[b][n] x[b][k]. One block per hidden
// unit n: warp w takes every 16th row from row w, lane l the inputs k = l and l + 32 (n_in <= 64);
// the 16 warps' partial sums are added in a fixed order.
__global__ void __launch_bounds__(512) k_layer1_grad(int64_t B, int n_in, int width, const float *__restrict__ x,
                                                     const bf16 *__restrict__ dZ, float *dW) {
  __shared__ float red[16][64];
  const int n = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float s0 = 0.f, s1 = 0.f;
  for (int64_t b = w; b < B; b += 16) {
    const float d = __bfloat162float(dZ[b * width + n]);
    if (lane < n_in) s0 = fmaf(d, x[b * n_in + lane], s0);
    if (lane + 32 < n_in) s1 = fmaf(d, x[b * n_in + lane + 32], s1);
  }
  red[w][lane] = s0;
  red[w][lane + 32] = s1;
  __syncthreads();
  if (threadIdx.x < n_in) {
    float s = 0.f;
    for (int i = 0; i < 16; ++i) s += red[i][threadIdx.x];
    dW[static_cast<int64_t>(n) * n_in + threadIdx.x] = s;
  }
}

// Column sums (bias gradients): db[n] = sum_b dZ[b][n]. A block of 32 x 32 threads covers 32
// columns: thread (x, y) sums every 32nd row from row y of column x, then the 32 partial sums of a
// column are added in a fixed tree order.
__global__ void __launch_bounds__(1024) k_colsum(int64_t rows, int cols, const bf16 *__restrict__ dZ, float *db) {
  __shared__ float red[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int n = blockIdx.x * 32 + tx;
  float s = 0.f;
  if (n < cols)
    for (int64_t b = ty; b < rows; b += 32) s += __bfloat162float(dZ[b * cols + n]);
  red[ty][tx] = s;
  __syncthreads();
  for (int k = 16; k > 0; k >>= 1) {
    if (ty < k) red[ty][tx] += red[ty + k][tx];
    __syncthreads();
  }
  if (ty == 0 && n < cols) db[n] = red[0][tx];
}

// Loss and output gradient: loss terms m (Y - T)^2 and dY = bf16(2 m (Y - T) / (B O)) with the
// optional nonnegative weights m (all ones when absent); per-block loss partials.
__global__ void k_loss(int64_t n, float scale, const float *__restrict__ Y, const float *__restrict__ T,
                       const float *__restrict__ mask, bf16 *dY, float *partial) {
  __shared__ float red[256];
  float s = 0.f;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x; e < n; e += static_cast<int64_t>(gridDim.x) * 256) {
    const float d = Y[e] - T[e];
    const float md = mask ? mask[e] * d : d;
    dY[e] = __float2bfloat16(2.f * md * scale);
    s = fmaf(md, d, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// the loss: the per-block partials added by 256 threads, then a fixed tree
__global__ void __launch_bounds__(256) k_loss_final(int nblocks, float scale, const float *partial, float *loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < nblocks; i += 256) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] * scale;
}

__global__ void k_adamw(int64_t n, float lr, float b1, float b2, float eps, float wd, float bc1, float bc2,
                        float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / bc1, vh = vi / bc2;
  w[i] = w[i] - lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
}

__global__ void k_to_bf16(int64_t n, const float *__restrict__ a, bf16 *b) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

// Ensemble estimate: preds [K][B][O] -> mean [B][O], err[b] = ln(10) * sqrt(mean_o var_k),
// the relative error of the spectrum implied by the models' spread of log10 predictions.
// Ensemble mean of log10 predictions and the relative L2 spectrum error implied by the models'
// spread: with mu_o the mean, var_o the unbiased variance over models and s_o = 10^mu_o,
// err = ln(10) sqrt(sum_o s_o^2 var_o / sum_o s_o^2) (first order in the log-space spread).
__global__ void k_ensemble(int K, int64_t B, int O, const float *__restrict__ preds, float *mean, float *err) {
  __shared__ float red[256];
  __shared__ float red2[256];
  const int64_t b = blockIdx.x;
  float mx = -INFINITY;
  for (int o = threadIdx.x; o < O; o += 256) {
    float s = 0.f;
    for (int k = 0; k < K; ++k) s += preds[(static_cast<int64_t>(k) * B + b) * O + o];
    const float mu = s / K;
    mean[b * O + o] = mu;
    mx = fmaxf(mx, mu);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + k]);
    __syncthreads();
  }
  mx = red[0];
  __syncthreads();
  float aw = 0.f, an = 0.f;
  for (int o = threadIdx.x; o < O; o += 256) {
    const float mu = mean[b * O + o];
    float v = 0.f;
    for (int k = 0; k < K; ++k) {
      const float d = preds[(static_cast<int64_t>(k) * B + b) * O + o] - mu;
      v = fmaf(d, d, v);
    }
    v = K > 1 ? v / (K - 1) : 0.f;
    const float w = exp10f(2.f * (mu - mx));  // (s_o / max s)^2
    aw = fmaf(w, v, aw);
    an += w;
  }
  red[threadIdx.x] = aw;
  red2[threadIdx.x] = an;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      red[threadIdx.x] += red[threadIdx.x + k];
      red2[threadIdx.x] += red2[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) err[b] = 2.302585093f * sqrtf(red2[0] > 0.f ? red[0] / red2[0] : 0.f);
}

// Label transform: out = log10(max(v, floor)) (FP64 in, FP32 out)
__global__ void k_log_targets(int64_t n, double floor_v, const double *__restrict__ v, float *out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = static_cast<float>(log10(fmax(v[i], floor_v)));
}

// Per-column mean and standard deviation of y [rows][cols] (FP64 accumulation).
__global__ void k_colstats(int64_t rows, int cols, const float *__restrict__ y, float *mean, float *stdv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0, s2 = 0.0;
  for (int64_t r = 0; r < rows; ++r) {
    const double v = y[r * cols + c];
    s += v;
    s2 += v * v;
  }
  const double mu = rows > 0 ? s / rows : 0.0;
  const double var = rows > 1 ? (s2 - rows * mu * mu) / (rows - 1) : 0.0;
  mean[c] = static_cast<float>(mu);
  stdv[c] = static_cast<float>(sqrt(fmax(var, 1e-12)));
}

__global__ void k_standardize(int64_t rows, int cols, float *y, const float *mean, const float *stdv, int inverse) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int c = static_cast<int>(i % cols);
  y[i] = inverse ? y[i] * stdv[c] + mean[c] : (y[i] - mean[c]) / stdv[c];
}

inline unsigned nblk(int64_t n, int t = 256) { return static_cast<unsigned>((n + t - 1) / t); }

}  // namespace
}  // namespace rad

using namespace rad;

struct rad_mlp_s {
  int n_in = 0, width = 0, depth = 0, n_out = 0;
  int64_t max_batch = 0;
  int64_t n_params = 0;
  // parameter layout in the FP32 buffers: W1 [width][n_in], b1, then for l = 2..depth
  // W_l [width][width], b_l, then W_out [n_out][width], b_out
  std::vector<int64_t> w_off, b_off;  // per layer (depth + 1 layers)
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16 *wb = nullptr;                  // BF16 copy of all weights (same offsets)
  float *Z = nullptr;                  // pre-activations [depth][max_batch][width]
  bf16 *H = nullptr;                   // activations [depth][max_batch][width]
  bf16 *dZ = nullptr;                  // [2][max_batch][width] ping-pong
  float *Y = nullptr;                  // [max_batch][n_out]
  bf16 *dY = nullptr;                  // [max_batch][n_out]
  float *partial = nullptr;            // loss partials [1024]
  float *splitk = nullptr;             // split-K partial sums [kSplitWsFloats]
  int64_t step = 0;
};

namespace {

int64_t layer_in(const rad_mlp_s *h, int l) { return l == 0 ? h->n_in : h->width; }
int64_t layer_out(const rad_mlp_s *h, int l) { return l == h->depth ? h->n_out : h->width; }

cudaError_t forward_impl(rad_mlp h, const float *x, int64_t B, float *y_out, bool keep, cudaStream_t st) {
  const int W = h->width, D = h->depth, O = h->n_out;
  float *Z = keep ? h->Z : nullptr;
  k_layer1<<<nblk(B * W), 256, 0, st>>>(B, h->n_in, W, x, h->w + h->w_off[0], h->w + h->b_off[0], Z, h->H);
  cudaError_t e = cudaGetLastError();
  for (int l = 1; l < D && e == cudaSuccess; ++l) {
    const bf16 *Hin = h->H + static_cast<int64_t>(l - 1) * h->max_batch * W;
    EpiHidden epi{h->w + h->b_off[l], keep ? h->Z + static_cast<int64_t>(l) * h->max_batch * W : nullptr,
                  h->H + static_cast<int64_t>(l) * h->max_batch * W, W};
    e = gemm<true, true>(static_cast<int>(B), W, W, Hin, W, h->wb + h->w_off[l], W, epi, h->splitk, st);
  }
  if (e != cudaSuccess) return e;
  const bf16 *Hlast = h->H + static_cast<int64_t>(D - 1) * h->max_batch * W;
  EpiOut epo{h->w + h->b_off[D], y_out, O};
  return gemm<true, true>(static_cast<int>(B), O, W, Hlast, W, h->wb + h->w_off[D], W, epo, h->splitk, st);
}

cudaError_t backward_impl(rad_mlp h, const float *x, const float *target, const float *mask, int64_t B, float *loss,
                          cudaStream_t st) {
  const int W = h->width, D = h->depth, O = h->n_out;
  cudaError_t e = forward_impl(h, x, B, h->Y, true, st);
  if (e != cudaSuccess) return e;
  const int64_t n = B * O;
  int nb = static_cast<int>(std::min<int64_t>(1024, (n + 255) / 256));
  const float scale = 1.f / static_cast<float>(n);
  k_loss<<<nb, 256, 0, st>>>(n, scale, h->Y, target, mask, h->dY, h->partial);
  if (loss) k_loss_final<<<1, 256, 0, st>>>(nb, scale, h->partial, loss);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // output layer: dW_out = dY^T H_last, db_out = colsum(dY), dH = dY W_out
  const bf16 *Hlast = h->H + static_cast<int64_t>(D - 1) * h->max_batch * W;
  EpiStore gW{h->g + h->w_off[D], W};
  e = gemm<false, false>(O, W, static_cast<int>(B), h->dY, O, Hlast, W, gW, h->splitk, st);
  if (e != cudaSuccess) return e;
  k_colsum<<<nblk(O, 32), 1024, 0, st>>>(B, O, h->dY, h->g + h->b_off[D]);
  int cur = 0;
  {
    EpiGradAct ga{h->Z + static_cast<int64_t>(D - 1) * h->max_batch * W, h->dZ, W};
    e = gemm<true, false>(static_cast<int>(B), W, O, h->dY, O, h->wb + h->w_off[D], W, ga, h->splitk, st);
    if (e != cudaSuccess) return e;
  }
  for (int l = D - 1; l >= 1; --l) {
    const bf16 *dZl = h->dZ + static_cast<int64_t>(cur) * h->max_batch * W;
    const bf16 *Hin = h->H + static_cast<int64_t>(l - 1) * h->max_batch * W;
    EpiStore gw{h->g + h->w_off[l], W};
    e = gemm<false, false>(W, W, static_cast<int>(B), dZl, W, Hin, W, gw, h->splitk, st);
    if (e != cudaSuccess) return e;
    k_colsum<<<nblk(W, 32), 1024, 0, st>>>(B, W, dZl, h->g + h->b_off[l]);
    bf16 *dZn = h->dZ + static_cast<int64_t>(cur ^ 1) * h->max_batch * W;
    EpiGradAct ga{h->Z + static_cast<int64_t>(l - 1) * h->max_batch * W, dZn, W};
    e = gemm<true, false>(static_cast<int>(B), W, W, dZl, W, h->wb + h->w_off[l], W, ga, h->splitk, st);
    if (e != cudaSuccess) return e;
    cur ^= 1;
  }
  const bf16 *dZ1 = h->dZ + static_cast<int64_t>(cur) * h->max_batch * W;
  k_layer1_grad<<<static_cast<unsigned>(W), 512, 0, st>>>(B, h->n_in, W, x, dZ1, h->g + h->w_off[0]);
  k_colsum<<<nblk(W, 32), 1024, 0, st>>>(B, W, dZ1, h->g + h->b_off[0]);
  return cudaGetLastError();
}

void mlp_free(rad_mlp h) {
  if (!h) return;
  cudaFree(h->w);
  cudaFree(h->g);
  cudaFree(h->m);
  cudaFree(h->v);
  cudaFree(h->wb);
  cudaFree(h->Z);
  cudaFree(h->H);
  cudaFree(h->dZ);
  cudaFree(h->Y);
  cudaFree(h->dY);
  cudaFree(h->partial);
  cudaFree(h->splitk);
  delete h;
}

}  // namespace

extern "C" {

int rad_mlp_create(int n_in, int width, int depth, int n_out, int64_t max_batch, uint64_t seed, rad_mlp *out) {
  if (!out || n_in < 1 || width < 1 || depth < 1 || n_out < 1 || max_batch < 1) return RAD_EINVAL;
  if (width % 2 || n_out % 2 || width > 8192 || n_out > (1 << 16) || n_in > 64) return RAD_EINVAL;
  if (max_batch > 64 * 65535) return RAD_EINVAL;  // GEMM grid y = batch rows / 64
  *out = nullptr;
  rad_mlp h = new rad_mlp_s();
  h->n_in = n_in;
  h->width = width;
  h->depth = depth;
  h->n_out = n_out;
  h->max_batch = max_batch;
  int64_t off = 0;
  for (int l = 0; l <= depth; ++l) {
    h->w_off.push_back(off);
    off += layer_in(h, l) * layer_out(h, l);
    h->b_off.push_back(off);
    off += layer_out(h, l);
  }
  h->n_params = off;
  const size_t pb = sizeof(float) * off;
  bool ok = cudaMalloc(&h->w, pb) == cudaSuccess && cudaMalloc(&h->g, pb) == cudaSuccess &&
            cudaMalloc(&h->m, pb) == cudaSuccess && cudaMalloc(&h->v, pb) == cudaSuccess &&
            cudaMalloc(&h->wb, sizeof(bf16) * off) == cudaSuccess &&
            cudaMalloc(&h->Z, sizeof(float) * depth * max_batch * width) == cudaSuccess &&
            cudaMalloc(&h->H, sizeof(bf16) * depth * max_batch * width) == cudaSuccess &&
            cudaMalloc(&h->dZ, sizeof(bf16) * 2 * max_batch * width) == cudaSuccess &&
            cudaMalloc(&h->Y, sizeof(float) * max_batch * n_out) == cudaSuccess &&
            cudaMalloc(&h->dY, sizeof(bf16) * max_batch * n_out) == cudaSuccess &&
            cudaMalloc(&h->partial, sizeof(float) * 1024) == cudaSuccess &&
            cudaMalloc(&h->splitk, sizeof(float) * kSplitWsFloats) == cudaSuccess;
  if (!ok) {
    mlp_free(h);
    return RAD_ENOMEM;
  }
  // initialisation: weights uniform in +-1/sqrt(fan_in) (seeded), biases 0
  std::vector<float> hw(off, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l <= depth; ++l) {
    const double bound = 1.0 / std::sqrt(static_cast<double>(layer_in(h, l)));
    std::uniform_real_distribution<double> U(-bound, bound);
    for (int64_t i = 0; i < layer_in(h, l) * layer_out(h, l); ++i) hw[h->w_off[l] + i] = static_cast<float>(U(rng));
  }
  ok = cudaMemcpy(h->w, hw.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(h->m, 0, pb) == cudaSuccess && cudaMemset(h->v, 0, pb) == cudaSuccess &&
       cudaMemset(h->g, 0, pb) == cudaSuccess;
  if (ok) {
    k_to_bf16<<<nblk(off), 256>>>(off, h->w, h->wb);
    ok = cudaDeviceSynchronize() == cudaSuccess;
  }
  if (!ok) {
    mlp_free(h);
    return RAD_ECUDA;
  }
  *out = h;
  return RAD_OK;
}

int rad_mlp_destroy(rad_mlp h) {
  cudaDeviceSynchronize();
  mlp_free(h);
  return RAD_OK;
}

int64_t rad_mlp_num_params(rad_mlp h) { return h ? h->n_params : 0; }

int rad_mlp_forward(rad_mlp h, const float *x, int64_t batch, float *y, void *stream) {
  if (!h || !x || !y || batch < 0) return RAD_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int64_t b0 = 0; b0 < batch; b0 += h->max_batch) {
    const int64_t nb = std::min<int64_t>(h->max_batch, batch - b0);
    if (forward_impl(h, x + b0 * h->n_in, nb, y + b0 * h->n_out, false, st) != cudaSuccess) return RAD_ECUDA;
  }
  return RAD_OK;
}

int rad_mlp_backward(rad_mlp h, const float *x, const float *target, const float *mask, int64_t batch, float *loss,
                     void *stream) {
  if (!h || !x || !target || batch < 1 || batch > h->max_batch) return RAD_EINVAL;
  return backward_impl(h, x, target, mask, batch, loss, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? RAD_OK
             : RAD_ECUDA;
}

int rad_mlp_adamw(rad_mlp h, float lr, float beta1, float beta2, float eps, float weight_decay, void *stream) {
  if (!h || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return RAD_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->step += 1;
  const float bc1 = 1.f - powf(beta1, static_cast<float>(h->step));
  const float bc2 = 1.f - powf(beta2, static_cast<float>(h->step));
  k_adamw<<<nblk(h->n_params), 256, 0, st>>>(h->n_params, lr, beta1, beta2, eps, weight_decay, bc1, bc2, h->w, h->g,
                                             h->m, h->v);
  k_to_bf16<<<nblk(h->n_params), 256, 0, st>>>(h->n_params, h->w, h->wb);
  return cudaGetLastError() == cudaSuccess ? RAD_OK : RAD_ECUDA;
}

int rad_mlp_train_step(rad_mlp h, const float *x, const float *target, const float *mask, int64_t batch, float lr,
                       float weight_decay, float *loss, void *stream) {
  int rc = rad_mlp_backward(h, x, target, mask, batch, loss, stream);
  if (rc) return rc;
  return rad_mlp_adamw(h, lr, 0.9f, 0.999f, 1e-8f, weight_decay, stream);
}

int rad_mlp_get(rad_mlp h, int what, float *host_out) {
  if (!h || !host_out || what < 0 || what > 3) return RAD_EINVAL;
  const float *src = what == 0 ? h->w : what == 1 ? h->g : what == 2 ? h->m : h->v;
  return cudaMemcpy(host_out, src, sizeof(float) * h->n_params, cudaMemcpyDeviceToHost) == cudaSuccess ? RAD_OK
                                                                                                         : RAD_ECUDA;
}

int rad_mlp_set_params(rad_mlp h, const float *host_in) {
  if (!h || !host_in) return RAD_EINVAL;
  if (cudaMemcpy(h->w, host_in, sizeof(float) * h->n_params, cudaMemcpyHostToDevice) != cudaSuccess) return RAD_ECUDA;
  k_to_bf16<<<nblk(h->n_params), 256>>>(h->n_params, h->w, h->wb);
  return cudaDeviceSynchronize() == cudaSuccess ? RAD_OK : RAD_ECUDA;
}

int rad_mlp_ensemble_estimate(const float *preds, int n_models, int64_t batch, int n_out, float *mean, float *err,
                              void *stream) {
  if (!preds || !mean || !err || n_models < 1 || batch < 0 || n_out < 1) return RAD_EINVAL;
  if (batch == 0) return RAD_OK;
  k_ensemble<<<static_cast<unsigned>(batch), 256, 0, static_cast<cudaStream_t>(stream)>>>(n_models, batch, n_out,
                                                                                         preds, mean, err);
  return cudaGetLastError() == cudaSuccess ? RAD_OK : RAD_ECUDA;
}

int rad_log_targets(const double *values, int64_t n, double floor_value, float *out, void *stream) {
  if (!values || !out || n < 0 || !(floor_value > 0.0)) return RAD_EINVAL;
  if (n == 0) return RAD_OK;
  k_log_targets<<<nblk(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, floor_value, values, out);
  return cudaGetLastError() == cudaSuccess ? RAD_OK : RAD_ECUDA;
}

int rad_column_stats(const float *y, int64_t rows, int cols, float *mean, float *stdv, void *stream) {
  if (!y || !mean || !stdv || rows < 0 || cols < 1) return RAD_EINVAL;
  k_colstats<<<nblk(cols), 256, 0, static_cast<cudaStream_t>(stream)>>>(rows, cols, y, mean, stdv);
  return cudaGetLastError() == cudaSuccess ? RAD_OK : RAD_ECUDA;
}

int rad_standardize(float *y, int64_t rows, int cols, const float *mean, const float *stdv, int inverse,
                    void *stream) {
  if (!y || !mean || !stdv || rows < 0 || cols < 1) return RAD_EINVAL;
  if (rows == 0) return RAD_OK;
  k_standardize<<<nblk(rows * cols), 256, 0, static_cast<cudaStream_t>(stream)>>>(rows, cols, y, mean, stdv,
                                                                                 inverse ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? RAD_OK : RAD_ECUDA;
}

}  // extern "C"
