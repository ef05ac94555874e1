// Row a2 in the mixed-precision path: the truncated KL field (Sec. 2.2,
// Eq. KL-expansion-deterministic)
//   Z[s][cell] = sum_q phi_q(centroid) * (sqrt(lam_q) xi[s][q])
// as one dense contraction (cells x modes) . (modes x samples) on the fifth-
// generation tensor cores (tcgen05, accumulators in tensor memory).
//
// Precision: FP32 accuracy from TF32 products by the three-term split
// (a = a_hi + a_lo with a_hi = tf32(a), a_lo = a - a_hi exact in FP32):
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,
// each product in TF32 with FP32 accumulation; the dropped a_lo b_lo term and
// the TF32 truncation of the lo parts are O(2^-21) relative.  One CTA owns a
// tile of 128 cells x NT samples (NT a multiple of 32, <= 256) and loops over
// the modes in chunks of 32; per chunk the threads stage the split operands
// in shared memory (K-major rows of 128 bytes, 128-byte swizzle), one thread
// issues 4 k-steps x 3 MMAs of shape 128 x NT x 8 into the TMEM accumulator
// and commits them to an mbarrier that every thread waits on before the next
// chunk overwrites the operands.  The epilogue reads the accumulator with
// tcgen05.ld (warp w reads TMEM lanes 32w..32w+31 = the tile's cells) and
// writes Z in FP64, coalesced along the cells.
//
// The mode functions are separable (products of 1D eigenfunctions), so the A
// operand is formed on the fly from the per-axis tables; no cells x modes
// table is stored.  Every wait on the mbarrier is bounded: on timeout the CTA
// records the failure in *err, waits (bounded) for its MMAs, frees its tensor
// memory and returns.
#include <stdint.h>

#include "internal.cuh"

namespace mlmc {

namespace {

constexpr int TC_M = 128;          // cells per tile (TMEM lanes)
constexpr int TC_KC = 32;          // modes per chunk: 32 x 4 bytes = one 128-byte row
constexpr int TC_THREADS = 128;
constexpr long long TC_SPIN_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) of a K-major tile with 128-byte rows and the
// 128-byte swizzle (16-byte chunk index XOR row mod 8; tiles 1024-byte aligned).
__device__ __forceinline__ uint32_t sw128(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 2) ^ (row & 7)) & 7) << 4) + (k & 3) * 4);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t instr_desc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split(double v, float* hi, float* lo) {
  const float f = (float)v;
  const float h = tf32_hi(f);
  *hi = h;
  *lo = f - h;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared memory of one CTA (dynamic, 1024-byte aligned): A_hi, A_lo [128 rows],
// B_hi, B_lo [NT rows], each row 128 bytes.
struct TcSmem {
  uint32_t a_hi, a_lo, b_hi, b_lo, total;
};
__host__ __device__ inline TcSmem tc_smem(int nt) {
  TcSmem s;
  s.a_hi = 0;
  s.a_lo = TC_M * 128;
  s.b_hi = 2 * TC_M * 128;
  s.b_lo = s.b_hi + nt * 128;
  s.total = s.b_lo + nt * 128;
  return s;
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS)
kl_field_tc_kernel(LevelDesc lv, int M, int nt, const double* __restrict__ sqrt_lam,
                   const int* __restrict__ idx, const double* __restrict__ phx,
                   const double* __restrict__ phy, const double* __restrict__ phz,
                   const double* __restrict__ xi, int n, double* __restrict__ Z,
                   unsigned long long* err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  // align the operand tiles to 1024 bytes (the swizzle atom)
  unsigned char* sm = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const TcSmem L = tc_smem(nt);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t cell0 = (int64_t)blockIdx.x * TC_M;
  const int s0 = blockIdx.y * nt;
  const uint32_t ncols = nt <= 32 ? 32u : nt <= 64 ? 64u : nt <= 128 ? 128u : 256u;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t bar = smem_addr(&mbar);
  const uint32_t idesc = instr_desc(nt);

  // this thread's cell for the A operand rows
  int ci[TC_M / TC_THREADS], cj[TC_M / TC_THREADS], ck[TC_M / TC_THREADS];
  bool cv[TC_M / TC_THREADS];
  for (int q = 0; q < TC_M / TC_THREADS; ++q) {
    const int64_t cell = cell0 + tid + q * TC_THREADS;
    cv[q] = cell < lv.cells;
    const int64_t c = cv[q] ? cell : 0;
    ci[q] = (int)(c % lv.n[0]);
    const int64_t r = c / lv.n[0];
    cj[q] = (int)(r % lv.n[1]);
    ck[q] = (int)(r / lv.n[1]);
  }

  bool ok = true;
  uint32_t phase = 0;
  const int chunks = (M + TC_KC - 1) / TC_KC;
  for (int ch = 0; ch < chunks && ok; ++ch) {
    const int q0 = ch * TC_KC;
    // A: row = cell of the tile, k = mode q0 + k (zero beyond M or the grid)
    for (int q = 0; q < TC_M / TC_THREADS; ++q) {
      const int row = tid + q * TC_THREADS;
      for (int k = 0; k < TC_KC; ++k) {
        const int mode = q0 + k;
        double v = 0.0;
        if (cv[q] && mode < M) {
          v = phx[(int64_t)idx[3 * mode] * lv.n[0] + ci[q]];
          if (lv.dim >= 2) v *= phy[(int64_t)idx[3 * mode + 1] * lv.n[1] + cj[q]];
          if (lv.dim >= 3) v *= phz[(int64_t)idx[3 * mode + 2] * lv.n[2] + ck[q]];
        }
        float hi, lo;
        split(v, &hi, &lo);
        *(float*)(sm + L.a_hi + sw128(row, k)) = hi;
        *(float*)(sm + L.a_lo + sw128(row, k)) = lo;
      }
    }
    // B: row = sample of the tile, k = mode; sqrt(lam) folded in
    for (int e = tid; e < nt * TC_KC; e += TC_THREADS) {
      const int row = e / TC_KC, k = e % TC_KC;
      const int s = s0 + row, mode = q0 + k;
      const double v = (s < n && mode < M) ? sqrt_lam[mode] * xi[(int64_t)s * M + mode] : 0.0;
      float hi, lo;
      split(v, &hi, &lo);
      *(float*)(sm + L.b_hi + sw128(row, k)) = hi;
      *(float*)(sm + L.b_lo + sw128(row, k)) = lo;
    }
    // make the generic-proxy stores visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t base = smem_addr(sm);
      for (int ks = 0; ks < TC_KC / 8; ++ks) {
        const uint32_t koff = ks * 32;   // 8 TF32 values = 32 bytes along the row
        const uint64_t ah = smem_desc(base + L.a_hi + koff), al = smem_desc(base + L.a_lo + koff);
        const uint64_t bh = smem_desc(base + L.b_hi + koff), bl = smem_desc(base + L.b_lo + koff);
        const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
        mma_tf32(tmem, ah, bh, idesc, first);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
          : "memory");
    }
    ok = mbar_wait(bar, phase);
    phase ^= 1u;
    ok = __syncthreads_and(ok);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");

  if (ok) {
    // epilogue: warp w owns TMEM lanes (tile rows) 32w .. 32w+31
    const int row = warp * 32 + lane;
    const int64_t cell = cell0 + row;
    for (int c0 = 0; c0 < nt; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (cell < lv.cells) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int s = s0 + c0 + c;
          if (s < n) Z[(int64_t)s * lv.cells + cell] = (double)v[c];
        }
      }
    }
  } else if (tid == 0) {
    atomicAdd(err, 1ull);
    // bounded wait for the MMAs already issued (the commit whose wait ran out;
    // phase was toggled after it) before the tensor memory is freed
    mbar_wait(bar, phase ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

size_t kl_tc_smem_bytes(int nt) { return tc_smem(nt).total + 1024; }

// Allows the largest tile's shared memory on the current device (once per
// context, before any launch or stream capture).
cudaError_t preload_kl_tc() {
  return cudaFuncSetAttribute(kl_field_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kl_tc_smem_bytes(256));
}

cudaError_t launch_kl_field_tc(const LevelDesc& lv, int M, const double* sqrt_lam, const int* idx,
                               const double* phi_x, const double* phi_y, const double* phi_z,
                               const double* xi, int n, double* Z, unsigned long long* err,
                               cudaStream_t st) {
  if (n == 0 || lv.cells == 0) return cudaSuccess;
  // samples per tile: the batch rounded up to 32, at most 256
  int nt = ((n + 31) / 32) * 32;
  if (nt > 256) nt = 256;
  const size_t smem = kl_tc_smem_bytes(nt);   // within the limit set by preload_kl_tc
  const int64_t tiles = (lv.cells + TC_M - 1) / TC_M;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  dim3 grid((unsigned)tiles, (unsigned)((n + nt - 1) / nt));
  kl_field_tc_kernel<<<grid, TC_THREADS, smem, st>>>(lv, M, nt, sqrt_lam, idx, phi_x, phi_y, phi_z,
                                                     xi, n, Z, err);
  return cudaGetLastError();
}

}  // namespace mlmc
