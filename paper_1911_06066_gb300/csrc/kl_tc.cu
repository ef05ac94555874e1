// Row a2 in the mixed-precision path: the truncated KL field (Sec. 3.1.1,
// Eq. KL-expansion-deterministic)
//   Z[s][cell] = sum_q phi_q(centroid) * (sqrt(lam_q) xi[s][q])
// as one dense contraction (cells x modes) . (modes x samples) on the fifth-
// generation tensor cores (tcgen05, accumulators in tensor memory).
//
// Precision: FP32 accuracy from TF32 products by the three-term split
// (a = a_hi + a_lo with a_hi = tf32(a), a_lo = a - a_hi exact in FP32):
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,
// each product in TF32 with FP32 accumulation; the dropped a_lo b_lo term and
// the TF32 truncation of the lo parts are O(2^-21) relative.
//
// Two kernels per call.  kl_tc_prep_kernel forms the B operand once:
// sqrt(lam_q) xi[s][q], split into hi / lo, written as the exact shared-memory
// image of every (sample tile, 32-mode chunk): K-major rows of 128 bytes with
// the 128-byte swizzle.  kl_field_tc_kernel: one CTA owns 128 cells x NT
// samples (NT a multiple of 32, <= 256) and runs a two-stage pipeline over the
// 32-mode chunks: one thread copies the chunk's B image into shared memory
// with cp.async.bulk (completion counted on a 'full' mbarrier), all threads
// form the A operand (the separable mode functions phi_x phi_y phi_z at the
// cells, FP32 tables) and split it, one thread issues 4 k-steps x 3 MMAs of
// shape 128 x NT x 8 into the TMEM accumulator and commits them to the
// stage's 'done' mbarrier, which the threads wait on before they refill that
// stage two chunks later -- so staging of chunk c+1 overlaps the MMAs of
// chunk c.  (With an explicit FP32 mode table -- the paper's KL variant --
// the A operand is read from it instead of the separable 1D tables.)  The
// epilogue reads the accumulator with tcgen05.ld (warps w and
// w+4 read TMEM lanes 32(w%4).. = the tile's cells, half the columns each)
// and writes Z in FP64, coalesced along the cells.
//
// Every wait is bounded: on timeout the CTA records the failure in *err,
// waits (bounded) for its outstanding MMAs, frees its tensor memory and
// returns.
#include <stdint.h>

#include "internal.cuh"

namespace mlmc {

namespace {

constexpr int TC_M = 128;          // cells per tile (TMEM lanes)
constexpr int TC_KC = 32;          // modes per chunk: 32 x 4 bytes = one 128-byte row
constexpr int TC_THREADS = 256;
constexpr long long TC_SPIN_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) of a K-major tile with 128-byte rows and the
// 128-byte swizzle (16-byte chunk index XOR row mod 8; tiles 1024-byte aligned).
__host__ __device__ __forceinline__ uint32_t sw128(int row, int k) {
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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = TC_SPIN_LIMIT) {
  for (long long it = 0; it < limit; ++it) {
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

// FP32 -> FP64 widening with integer operations (exact): a normal float's
// exponent is rebiased (+1023-127) and its mantissa shifted into place; zeros
// keep their sign; other encodings (subnormal, inf, nan -- not produced for a
// KL field) take the conversion instruction, which runs on the FP64 pipe.
__device__ __forceinline__ double widen(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e - 1u < 254u) {
    const uint64_t d = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(e + 896u) << 52) |
                       ((uint64_t)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
  }
  if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((uint64_t)b << 32));
  return (double)f;
}

// Shared memory of one CTA (dynamic, 1024-byte aligned), per stage:
// A_hi, A_lo [128 rows], B_hi, B_lo [NT rows], each row 128 bytes.
struct TcSmem {
  uint32_t a_hi[2], a_lo[2], b_hi[2], b_lo[2], total;
};
__host__ __device__ inline TcSmem tc_smem(int nt) {
  TcSmem s;
  uint32_t o = 0;
  for (int st = 0; st < 2; ++st) {
    s.a_hi[st] = o; o += TC_M * 128;
    s.a_lo[st] = o; o += TC_M * 128;
    s.b_hi[st] = o; o += nt * 128;
    s.b_lo[st] = o; o += nt * 128;
  }
  s.total = o;
  return s;
}

// Layout of the prepared B operand: for sample tile t and chunk c, the hi image
// (nt rows x 128 bytes) then the lo image; bytes per tile-chunk 2 nt 128.
__host__ __device__ inline int64_t bprep_offset(int t, int c, int chunks, int nt) {
  return ((int64_t)t * chunks + c) * 2 * nt * 128;
}

}  // namespace

// One thread per (sample slot of the padded batch, mode slot of the padded
// mode range): v = sqrt(lam_q) xi[s][q] in FP64 (0 outside the batch or the
// modes), split into TF32 hi and FP32 lo, stored in the swizzled images.
__global__ void kl_tc_prep_kernel(int M, int n, int nt, int chunks, const double* __restrict__ sqrt_lam,
                                  const double* __restrict__ xi, unsigned char* __restrict__ bprep) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int kpad = chunks * TC_KC;
  const int tiles = (n + nt - 1) / nt;
  if (g >= (int64_t)tiles * nt * kpad) return;
  const int s = (int)(g / kpad), q = (int)(g % kpad);
  const double v = (s < n && q < M) ? sqrt_lam[q] * xi[(int64_t)s * M + q] : 0.0;
  const float f = (float)v;
  const float hi = tf32_hi(f);
  const int t = s / nt, row = s % nt, c = q / TC_KC, k = q % TC_KC;
  unsigned char* img = bprep + bprep_offset(t, c, chunks, nt);
  *(float*)(img + sw128(row, k)) = hi;
  *(float*)(img + nt * 128 + sw128(row, k)) = f - hi;
}

__global__ void __launch_bounds__(TC_THREADS)
kl_field_tc_kernel(LevelDesc lv, int M, int nt, const int* __restrict__ idx,
                   const float* __restrict__ phx, const float* __restrict__ phy,
                   const float* __restrict__ phz, const float* __restrict__ phi_cells,
                   const unsigned char* __restrict__ bprep, int n, double* __restrict__ Z,
                   unsigned long long* err, long long check_limit) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  // align the operand tiles to 1024 bytes (the swizzle atom)
  unsigned char* sm = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[2], done[2];
  __shared__ uint32_t tmem_slot;
  const TcSmem L = tc_smem(nt);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t cell0 = (int64_t)blockIdx.x * TC_M;
  const int tile = blockIdx.y, s0 = tile * nt;
  const uint32_t ncols = nt <= 32 ? 32u : nt <= 64 ? 64u : nt <= 128 ? 128u : 256u;
  const int chunks = (M + TC_KC - 1) / TC_KC;
  const uint32_t bbytes = (uint32_t)nt * 128;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int st = 0; st < 2; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[st])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&done[st])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = instr_desc(nt);
  const uint32_t base = smem_addr(sm);

  // A operand rows: this thread forms row (tid % 128), modes [16 h, 16 h + 16)
  // of every chunk, h = tid / 128
  const int arow = tid & (TC_M - 1), ahalf = tid >> 7;
  const int64_t acell = cell0 + arow;
  const bool avalid = acell < lv.cells;
  int ai = 0, aj = 0, ak = 0;
  if (avalid) {
    ai = (int)(acell % lv.n[0]);
    const int64_t r = acell / lv.n[0];
    aj = (int)(r % lv.n[1]);
    ak = (int)(r / lv.n[1]);
  }

  bool ok = true;
  int issued = 0;     // chunks whose MMAs were committed
  int stuck = -1;     // chunk whose operand copy did not land in time
  if (check_limit >= 0) {
    // Check of the bounded-wait path: before any copy or MMA of this CTA is
    // issued, wait at most check_limit polls on the first stage's 'full'
    // barrier, which nothing has armed yet -- the wait runs out, nothing is
    // in flight, and the CTA takes the timeout exit below.
    if (tid == 0) ok = mbar_wait(smem_addr(&full[0]), 0u, check_limit);
    ok = __syncthreads_and(ok);
  }
  for (int c = 0; c < chunks && ok; ++c) {
    const int st = c & 1;
    if (c >= 2) ok = mbar_wait(smem_addr(&done[st]), (uint32_t)(((c - 2) >> 1) & 1));
    ok = __syncthreads_and(ok);
    if (!ok) break;
    if (tid == 0) {
      const uint32_t fb = smem_addr(&full[st]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(2 * bbytes)
                   : "memory");
      const unsigned char* src = bprep + bprep_offset(tile, c, chunks, nt);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              base + L.b_hi[st]),
          "l"(src), "r"(bbytes), "r"(fb)
          : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              base + L.b_lo[st]),
          "l"(src + bbytes), "r"(bbytes), "r"(fb)
          : "memory");
    }
    // A: the chunk's 32 modes at this thread's cell, split
    for (int kk = 0; kk < TC_KC / 2; ++kk) {
      const int k = ahalf * (TC_KC / 2) + kk;
      const int mode = c * TC_KC + k;
      float v = 0.f;
      if (avalid && mode < M) {
        if (phi_cells) {
          v = phi_cells[acell * M + mode];    // explicit mode table (the paper's KL)
        } else {
          v = phx[(int64_t)idx[3 * mode] * lv.n[0] + ai];
          if (lv.dim >= 2) v *= phy[(int64_t)idx[3 * mode + 1] * lv.n[1] + aj];
          if (lv.dim >= 3) v *= phz[(int64_t)idx[3 * mode + 2] * lv.n[2] + ak];
        }
      }
      const float h = tf32_hi(v);
      *(float*)(sm + L.a_hi[st] + sw128(arow, k)) = h;
      *(float*)(sm + L.a_lo[st] + sw128(arow, k)) = v - h;
    }
    // make the generic-proxy stores visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      bool landed = mbar_wait(smem_addr(&full[st]), (uint32_t)((c >> 1) & 1));
      if (landed) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int ks = 0; ks < TC_KC / 8; ++ks) {
          const uint32_t koff = ks * 32;   // 8 TF32 values = 32 bytes along the row
          const uint64_t ah = smem_desc(base + L.a_hi[st] + koff);
          const uint64_t al = smem_desc(base + L.a_lo[st] + koff);
          const uint64_t bh = smem_desc(base + L.b_hi[st] + koff);
          const uint64_t bl = smem_desc(base + L.b_lo[st] + koff);
          const uint32_t acc = (c == 0 && ks == 0) ? 0u : 1u;
          mma_tf32(tmem, ah, bh, idesc, acc);
          mma_tf32(tmem, ah, bl, idesc, 1u);
          mma_tf32(tmem, al, bh, idesc, 1u);
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&done[st]))
            : "memory");
      } else {
        ok = false;
        stuck = c;
      }
    }
    ok = __syncthreads_and(ok);
    if (ok) issued = c + 1;
  }
  // the last commit completes after every earlier MMA of this CTA
  if (ok && issued > 0) {
    const int c = issued - 1;
    ok = mbar_wait(smem_addr(&done[c & 1]), (uint32_t)((c >> 1) & 1));
    ok = __syncthreads_and(ok);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");

  if (ok) {
    // epilogue: warps w and w + 4 own TMEM lanes 32 (w % 4) .. (the tile's
    // cells); each takes half of the sample columns
    const int lw = warp & 3;
    const int row = lw * 32 + lane;
    const int64_t cell = cell0 + row;
    const int half = ((nt / 2 + 31) / 32) * 32;   // a multiple of 32 columns
    const int c_lo = (warp >> 2) * half, c_hi = c_lo + half < nt ? c_lo + half : nt;
    for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(lw * 32) << 16) + (uint32_t)c0, v);
      if (cell < lv.cells) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int s = s0 + c0 + q;
          if (s < n) Z[(int64_t)s * lv.cells + cell] = widen(v[q]);
        }
      }
    }
  } else if (tid == 0) {
    atomicAdd(err, 1ull);
    // bounded waits for the MMAs already committed before the memory is freed
    if (issued > 0) mbar_wait(smem_addr(&done[(issued - 1) & 1]), (uint32_t)(((issued - 1) >> 1) & 1));
    if (stuck >= 0) mbar_wait(smem_addr(&full[stuck & 1]), (uint32_t)((stuck >> 1) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

size_t kl_tc_smem_bytes(int nt) { return tc_smem(nt).total + 1024; }

// Samples per tile: the batch rounded up to 32, at most 256.
static int kl_tc_nt(int n) {
  int nt = ((n + 31) / 32) * 32;
  return nt > 256 ? 256 : nt;
}

// Bytes of the prepared B operand (256-byte multiple) for n samples, M modes.
size_t kl_tc_workspace_bytes(int M, int n) {
  if (n <= 0) return 0;
  const int nt = kl_tc_nt(n), tiles = (n + nt - 1) / nt, chunks = (M + TC_KC - 1) / TC_KC;
  return (size_t)(((int64_t)tiles * chunks * 2 * nt * 128 + 255) & ~(int64_t)255);
}

// Allows the largest tile's shared memory on the current device (once per
// context, before any launch or stream capture).
cudaError_t preload_kl_tc() {
  return cudaFuncSetAttribute(kl_field_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kl_tc_smem_bytes(256));
}

cudaError_t launch_kl_field_tc(const LevelDesc& lv, int M, const double* sqrt_lam, const int* idx,
                               const float* phi_x, const float* phi_y, const float* phi_z,
                               const float* phi_cells, const double* xi, int n, double* Z, void* ws,
                               unsigned long long* err, long long check_limit, cudaStream_t st) {
  if (n == 0 || lv.cells == 0) return cudaSuccess;
  const int nt = kl_tc_nt(n);
  const int chunks = (M + TC_KC - 1) / TC_KC, tiles = (n + nt - 1) / nt;
  const int64_t prep = (int64_t)tiles * nt * chunks * TC_KC;
  kl_tc_prep_kernel<<<(unsigned)((prep + 255) / 256), 256, 0, st>>>(M, n, nt, chunks, sqrt_lam, xi,
                                                                   (unsigned char*)ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = kl_tc_smem_bytes(nt);   // within the limit set by preload_kl_tc
  const int64_t mt = (lv.cells + TC_M - 1) / TC_M;
  if (mt > 0x7fffffff || tiles > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)mt, (unsigned)tiles);
  kl_field_tc_kernel<<<grid, TC_THREADS, smem, st>>>(lv, M, nt, idx, phi_x, phi_y, phi_z, phi_cells,
                                                     (const unsigned char*)ws, n, Z, err,
                                                     check_limit);
  return cudaGetLastError();
}

}  // namespace mlmc
