// Self-test of the tcgen05 building blocks (w2_umma.cuh) on one CTA: one
// D = A B tile through the shared-memory descriptors, the instruction
// descriptor, TMEM allocation, MMA issue, commit to an mbarrier (bounded
// wait), TMEM store and load.  TMEM is first filled with a marker word, then
// the MMA runs, then all 128 lanes of 2N columns are copied out, so that the
// caller sees which lanes and columns the MMA wrote as well as their values.
//
// Safety by construction: each operand sits in a zeroed shared-memory region
// larger than the farthest byte the MMA can address with the descriptor's
// two core-matrix strides taken either way round and with M or N read as
// twice their value (checked on the host before the launch); the CTA holds
// all 512 TMEM columns, so a wider write stays inside its allocation; the
// completion wait gives up after about a second and reports W2_ERR_TIMEOUT;
// the allocating warp always releases TMEM before the CTA ends.
#include <stdint.h>

#include "w2_internal.cuh"
#include "w2_umma.cuh"

namespace w2 {
namespace {

constexpr uint32_t kRegA = 96 * 1024, kRegB = 32 * 1024;
constexpr uint32_t kMarker = 0x7fc0deadu;

struct UTArgs {
  int M, N, K, a_mn, b_mn, swap;
  const uint16_t *A;  // M x K, row-major BF16 bits
  const uint16_t *B;  // K x N, row-major BF16 bits
  uint32_t *dump;     // [128][2N] TMEM words
};

__device__ int g_ut_status;

// Core-matrix strides of a tiled operand: K direction and M/N direction.
__host__ __device__ inline void strides(int R, int K, bool mn, uint32_t &sk, uint32_t &sr) {
  if (mn) {  // tile_off(k, r, R): rows along K
    sk = (uint32_t)(R / 8) * 128u;
    sr = 128u;
  } else {   // tile_off(r, k, K): rows along M/N
    sk = 128u;
    sr = (uint32_t)(K / 8) * 128u;
  }
}

// Start-address advance per K step of 16.
__host__ __device__ inline uint32_t kstep(int R, bool mn) { return mn ? 2u * (uint32_t)(R / 8) * 128u : 256u; }

__global__ void __launch_bounds__(128, 1) k_umma_selftest(UTArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *sA = sm, *sB = sm + kRegA;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + kRegA + kRegB);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + kRegA + kRegB + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (uint32_t i = tid; i < (kRegA + kRegB) / 16; i += 128) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int e = tid; e < a.M * a.K; e += 128) {
    const int m = e / a.K, k = e - m * a.K;
    const uint32_t off = a.a_mn ? umma::tile_off(k, m, a.M) : umma::tile_off(m, k, a.K);
    *reinterpret_cast<uint16_t *>(sA + off) = a.A[e];
  }
  for (int e = tid; e < a.K * a.N; e += 128) {
    const int k = e / a.N, n = e - k * a.N;
    const uint32_t off = a.b_mn ? umma::tile_off(k, n, a.N) : umma::tile_off(n, k, a.K);
    *reinterpret_cast<uint16_t *>(sB + off) = a.B[e];
  }
  umma::fence_proxy_async();
  if (warp == 0) {
    umma::tmem_alloc(slot, 512);
    umma::tmem_relinquish();
  }
  if (tid == 0) umma::mbar_init(mbar, 1);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tbase = *slot;
  const uint32_t lanes = (uint32_t)(32 * warp) << 16;

  uint32_t r[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) r[j] = kMarker;
  for (int c = 0; c < 2 * a.N; c += 16) umma::tmem_st16(tbase + lanes + (uint32_t)c, r);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();

  if (tid == 0) {
    uint32_t ska, sra, skb, srb;
    strides(a.M, a.K, a.a_mn, ska, sra);
    strides(a.N, a.K, a.b_mn, skb, srb);
    const uint32_t la = a.swap ? sra : ska, sa = a.swap ? ska : sra;
    const uint32_t lb = a.swap ? srb : skb, sb = a.swap ? skb : srb;
    const uint32_t idesc = umma::idesc_bf16(a.M, a.N, a.a_mn, a.b_mn);
    for (int kc = 0; kc < a.K / 16; ++kc) {
      const uint64_t ad = umma::smem_desc(umma::smem_u32(sA) + kc * kstep(a.M, a.a_mn), la, sa);
      const uint64_t bd = umma::smem_desc(umma::smem_u32(sB) + kc * kstep(a.N, a.b_mn), lb, sb);
      umma::mma_bf16(tbase, ad, bd, idesc, kc > 0 ? 1u : 0u);
    }
    umma::mma_commit(mbar);
  }
  __syncwarp();
  if (!umma::mbar_wait_bounded(mbar, 0, 2000000000ll) && lane == 0) atomicOr(&g_ut_status, 1);
  umma::fence_after();
  for (int c = 0; c < 2 * a.N; c += 16) {
    umma::tmem_ld16(tbase + lanes + (uint32_t)c, r);
#pragma unroll
    for (int j = 0; j < 16; ++j) a.dump[(size_t)(32 * warp + lane) * 2 * a.N + c + j] = r[j];
  }
  umma::fence_before();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, 512);
}

// Farthest byte (exclusive) an MMA sequence over one operand can address:
// R rows (along M or N) of which the hardware might read up to 2R, nk K
// steps, the two strides taken either way round.
uint32_t reach(int R, int K, bool mn) {
  uint32_t sk, sr;
  strides(R, K, mn, sk, sr);
  const uint32_t big = sk > sr ? sk : sr;
  const uint32_t groups = (uint32_t)(2 * R / 8);
  return (uint32_t)(K / 16 - 1) * kstep(R, mn) + (groups - 1) * big + big + 128u;
}

}  // namespace
}  // namespace w2

extern "C" uint64_t w2_debug_umma_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return w2::umma::smem_desc(saddr, lbo, sbo);
}

extern "C" uint32_t w2_debug_umma_idesc(int32_t M, int32_t N, int32_t a_mn, int32_t b_mn) {
  return w2::umma::idesc_bf16(M, N, a_mn != 0, b_mn != 0);
}

extern "C" uint32_t w2_debug_umma_tile_off(int32_t r, int32_t c, int32_t ncol) {
  return w2::umma::tile_off(r, c, ncol);
}

extern "C" w2_status w2_debug_umma_gemm(int32_t M, int32_t N, int32_t K, int32_t a_mn, int32_t b_mn, int32_t swap,
                                        const uint16_t *A, const uint16_t *B, uint32_t *dump) {
  using namespace w2;
  if (!A || !B || !dump || (M != 64 && M != 128) || !umma::shape_ok(M, N) || N > 64 || K < 16 || K > 64 ||
      K % 16)
    return W2_ERR_ARG;
  if (reach(M, K, a_mn != 0) > kRegA || reach(N, K, b_mn != 0) > kRegB) return W2_ERR_ARG;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return W2_ERR_CUDA;
  if (prop.major != 10) return W2_ERR_UNSUPPORTED;
  const size_t smem = kRegA + kRegB + 16;
  cudaError_t e = cudaFuncSetAttribute(k_umma_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int zero = 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_ut_status, &zero, sizeof(int));
  if (e != cudaSuccess) {
    note_cuda_error(e);
    return W2_ERR_CUDA;
  }
  UTArgs a{M, N, K, a_mn != 0, b_mn != 0, swap != 0, A, B, dump};
  k_umma_selftest<<<1, 128, smem>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&st, g_ut_status, sizeof(int));
  if (e != cudaSuccess) {
    note_cuda_error(e);
    return W2_ERR_CUDA;
  }
  return st ? W2_ERR_TIMEOUT : W2_OK;
}
