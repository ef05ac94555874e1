// Rows a4-a8 on thread-block clusters: the same per-sample Newton-CG sweep as
// solver.cu (Sec. 3.3, Eq. mono_disc; Sec. 3.5 -- the algorithm, its root
// selection rule and its stopping tests are documented there), laid out for
// GB300's distributed shared memory.
//
// Mapping.  One cluster of C CTAs owns one sample.  The node grid is cut into
// C bands of H whole rows (2D: rows of constant y; 3D: planes of constant z);
// CTA r owns rows [rH, min((r+1)H, rows)).  Every per-node vector of the sweep
// -- the FP64 state u (two slices) and residual F, the CG vectors r, z, p, q,
// d, diag, diag^-1 (FP64, or FP32 in the mixed path), and, when they fit, the
// couplings used by the CG in the CG's precision -- lives in the owning CTA's shared memory for
// the whole time sweep.  A stencil touching the row above or below the band
// reads the neighbour CTA's shared memory directly (DSMEM), so there is no
// halo copy; the barrier that publishes a vector is the one the algorithm
// needs anyway.  Dot products are reduced per warp, per CTA (fixed order),
// then across the cluster by reading every CTA's partial in rank order, so the
// result is identical on all CTAs and deterministic.  Per CG iteration the
// cluster synchronises twice (p^T H p and r^T z): the new search direction
// is formed inside the next stencil pass.
//
// Only the per-sample couplings (read once per Newton step by the residual)
// and the outputs stay in global memory.
//
// Large grids (the 3D levels) do not fit a cluster's shared memory.  For them
// the same kernel runs with its vectors in global memory (GM = true): each
// sample's vectors are contiguous, CTA r of the cluster owns the contiguous
// node range [rH, min((r+1)H, N)) (H nodes, not whole rows), a stencil reads
// its neighbours at constant offsets from the node, and the cluster barriers
// (release / acquire at cluster scope) publish each vector to the other CTAs.
// The reductions stay in shared memory and DSMEM.
//
// With MG (global-memory layout only) the CG is preconditioned by one V-cycle
// of the geometric multigrid of gmg.cuh instead of Jacobi: the Galerkin
// hierarchy is built once per sample before the time sweep, the coarse
// diagonal terms once per Newton iteration, and z = V(r) replaces z = r / |H_ii|.
#pragma once
#include <cooperative_groups.h>
#include <math.h>

#include "gmg.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace mlmc {

namespace {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Band geometry of this CTA.
struct Band {
  int C, rank, H, row0, row1, rowlen, nrows, nb, nmax;
  int N0, N1, N2;
  int base;   // first node of this CTA
};

// A per-node shared-memory vector and the same vector of the two neighbour
// CTAs (nullptr at the ends of the cluster).
template <typename T>
struct View {
  T* loc;
  const T* prev;
  const T* next;
};

template <bool GM, typename T>
__device__ __forceinline__ View<T> make_view(cg::cluster_group& cl, const Band& b, T* p) {
  View<T> v;
  v.loc = p;
  v.prev = !GM && b.rank > 0 ? cl.map_shared_rank(p, b.rank - 1) : nullptr;
  v.next = !GM && b.rank < b.C - 1 ? cl.map_shared_rank(p, b.rank + 1) : nullptr;
  return v;
}

// sum_o c[o] v[neighbour o] for the node (i, j, k); out-of-domain neighbours
// have zero couplings and are skipped.  c(o) returns the coupling.  With GM
// the vector is contiguous over the sample and v.loc points at node b.base.
template <int DIM, bool GM, typename TA, typename TV, typename CF>
__device__ __forceinline__ TA stencil_band(const Band& b, const View<TV>& v, int i, int j, int k,
                                           CF c) {
  TA y = 0;
#pragma unroll
  for (int o = 0; o < (DIM == 3 ? 27 : (DIM == 2 ? 9 : 3)); ++o) {
    const int dx = o % 3 - 1, dy = (DIM >= 2 ? (o / 3) % 3 - 1 : 0), dz = DIM == 3 ? o / 9 - 1 : 0;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    if (ii < 0 || ii >= b.N0 || jj < 0 || jj >= b.N1 || kk < 0 || kk >= b.N2) continue;
    const int row = DIM == 3 ? kk : jj;
    const int inrow = DIM == 3 ? jj * b.N0 + ii : ii;
    TV val;
    if (GM) val = v.loc[row * b.rowlen + inrow - b.base];
    else if (row >= b.row0 && row < b.row1) val = v.loc[(row - b.row0) * b.rowlen + inrow];
    else if (row < b.row0) val = v.prev[(b.H - 1) * b.rowlen + inrow];
    else val = v.next[inrow];
    y += (TA)c(o) * (TA)val;
  }
  return y;
}

// Neighbour sum for a node whose 3^dim neighbours all lie inside the domain
// and inside this CTA's band: constant local offsets.
template <int DIM, typename TA, typename TV, typename CF>
__device__ __forceinline__ TA stencil_fast(const TV* v, int a, int N0, int N01, CF c) {
  TA y = 0;
#pragma unroll
  for (int o = 0; o < (DIM == 3 ? 27 : (DIM == 2 ? 9 : 3)); ++o) {
    const int dx = o % 3 - 1, dy = (DIM >= 2 ? (o / 3) % 3 - 1 : 0), dz = DIM == 3 ? o / 9 - 1 : 0;
    y += (TA)c(o) * (TA)v[a + dx + dy * N0 + dz * N01];
  }
  return y;
}

// Synchronisation of the group layout (GRP): the G CTAs of one sample are
// not a hardware cluster but CTAs of an ordinary grid that took consecutive
// tickets on arrival (so a group only ever waits for CTAs that are already
// resident).  A barrier is a monotonic arrival counter in global memory:
// every CTA adds one and waits until the counter reaches G times the number
// of barriers passed.  Thread 0 publishes the CTA's writes with a gpu-scope
// fence before arriving and acquires the others' after the wait, between two
// CTA barriers -- the order in which grid-wide barriers are built.  A wait is
// bounded (GROUP_WAIT_NS of global time); a CTA whose wait runs out raises
// the sample's give-up flag, which ends every other wait of the sample at
// once, and the kernel reports MLMC_ERR_TIMEOUT for the sample.
constexpr unsigned long long GROUP_WAIT_NS = 180ull * 1000000000ull;

struct GroupSync {
  unsigned* ctr = nullptr;    // arrivals of the sample's CTAs
  unsigned* flag = nullptr;   // give-up flag of the sample
  double* slot = nullptr;     // reduction partials [2][8][G]
  unsigned target = 0;        // arrivals that complete the next barrier
  int* abort = nullptr;       // shared: this CTA gave up
  long long check = -1;       // >= 0: wait for one arrival more, at most check polls
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __noinline__ void group_barrier(GroupSync& gs, int G) {
  __syncthreads();
  if (threadIdx.x == 0) {
    gs.target += (unsigned)G;
    __threadfence();
    atomicAdd(gs.ctr, 1u);
    if (*gs.abort == 0) {
      const unsigned long long t0 = global_ns();
      const unsigned want = gs.target + (gs.check >= 0 ? 1u : 0u);   // the check never arrives
      long long polls = 0;
      while ((int)(ld_acquire_gpu(gs.ctr) - want) < 0) {
        ++polls;
        if (ld_acquire_gpu(gs.flag) != 0u || (gs.check >= 0 && polls > gs.check) ||
            ((polls & 255) == 0 && global_ns() - t0 > GROUP_WAIT_NS)) {
          *gs.abort = 1;
          atomicExch(gs.flag, 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

__device__ __forceinline__ void cluster_barrier(cg::cluster_group& cl, int C) {
  if (C == 1) __syncthreads(); else cl.sync();
}

template <bool GRP>
__device__ __forceinline__ void sync_all(cg::cluster_group& cl, int C, GroupSync& gs) {
  if (GRP) group_barrier(gs, C);
  else cluster_barrier(cl, C);
}

// Coupling o of node A from per-sample arrays with N nodes per offset.  SYM
// (3D global-memory sweeps): each symmetric pair is stored once, offsets
// 13..26 at 0..13, and offset o < 13 is the neighbour A + off(o)'s entry
// 26 - o (at 13 - o); o is a constant after unrolling, so is the branch.
template <bool SYM, int DIM, typename T>
__device__ __forceinline__ T coupling(const T* c, int o, int64_t N, int A, int N0, int N01) {
  constexpr int CTR = DIM == 3 ? 13 : (DIM == 2 ? 4 : 1);
  if (!SYM) return c[(int64_t)o * N + A];
  if (o >= CTR) return c[(int64_t)(o - CTR) * N + A];
  const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
  return c[(int64_t)(CTR - o) * N + A + dx + dy * N0 + dz * N01];
}

// The neighbour sum of the node with packed code c (i | j << 11 | k << 22,
// bit 31: every neighbour inside the domain and the band).  Shared-memory
// bands: the constant-offset sum or the band-aware one.  Global-memory layouts
// (GM, pred): one branch-free unrolled sum for every node, each offset
// predicated on the neighbour lying inside the domain -- the same terms in the
// same order as the other two, without a warp running both paths where its
// nodes straddle a boundary (chosen per level: SolverParams::pred_stencil).
template <int DIM, bool GM, typename TA, typename TV, typename CF>
__device__ __forceinline__ TA stencil_node(const Band& b, const TV* vloc, const View<TV>& v, int a,
                                           unsigned c, int N01, CF cf, int pred) {
  const int i = (int)(c & 2047u), j = (int)((c >> 11) & 2047u), k = (int)((c >> 22) & 511u);
  if (!GM || !pred) {
    return (c & 0x80000000u) ? stencil_fast<DIM, TA>(vloc, a, b.N0, N01, cf)
                             : stencil_band<DIM, GM, TA>(b, v, i, j, k, cf);
  }
  const bool xl = i > 0, xh = i < b.N0 - 1;
  const bool yl = DIM < 2 || j > 0, yh = DIM < 2 || j < b.N1 - 1;
  const bool zl = DIM < 3 || k > 0, zh = DIM < 3 || k < b.N2 - 1;
  TA y = 0;
#pragma unroll
  for (int o = 0; o < (DIM == 3 ? 27 : (DIM == 2 ? 9 : 3)); ++o) {
    const int dx = o % 3 - 1, dy = (DIM >= 2 ? (o / 3) % 3 - 1 : 0), dz = DIM == 3 ? o / 9 - 1 : 0;
    const bool in = (dx < 0 ? xl : (dx > 0 ? xh : true)) && (dy < 0 ? yl : (dy > 0 ? yh : true)) &&
                    (dz < 0 ? zl : (dz > 0 ? zh : true));
    if (in) y += (TA)cf(o) * (TA)vloc[a + dx + dy * b.N0 + dz * N01];
  }
  return y;
}

// Deterministic cluster-wide sums (op 0) or maxima (op 1, of non-negative
// values) of K values per thread.  Warps reduce by butterfly shuffles in TP
// (float in the mixed CG, double otherwise); warp 0 combines the CTA's warps
// by a fixed shuffle tree; lane q then stores the CTA's K partials into
// CTA q's slot[par][k][rank] (remote stores in parallel), one cluster barrier
// publishes them, and warp 0 of every CTA combines the C partials by the same
// fixed tree -- so every CTA obtains identical totals.  Lane 0 writes the
// totals to bc[0..K) and calls post(bc) to derive further scalars in bc[K..8).
// Every thread reads bc[] after the call returns.
template <typename TP>
__device__ __forceinline__ TP combine(TP x, TP y, int op) { return op ? (x > y ? x : y) : x + y; }

template <int NT, typename TP, int K, bool GRP, typename POST>
__device__ __forceinline__ void cluster_reduce(TP (&v)[K], int op, double* red, double* slot,
                                               double* bc, int& par, cg::cluster_group& cl, int C,
                                               int rank, GroupSync& gs, POST post) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = combine(v[k], __shfl_xor_sync(0xffffffffu, v[k], o), op);
    if (lane == 0) red[k * 32 + warp] = (double)v[k];
  }
  __syncthreads();
  if (warp == 0) {
    TP t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      t[k] = lane < NT / 32 ? (TP)red[k * 32 + lane] : (TP)0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t[k] = combine(t[k], __shfl_xor_sync(0xffffffffu, t[k], o), op);
    }
    if (GRP) {
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) gs.slot[(par * 8 + k) * C + rank] = (double)t[k];
      }
    } else if (C == 1) {
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) bc[k] = (double)t[k];
        post(bc);
      }
    } else if (lane < C) {
      double* dst = cl.map_shared_rank(slot + par * 64 + rank, lane);
#pragma unroll
      for (int k = 0; k < K; ++k) dst[k * 16] = (double)t[k];
    }
  }
  if (GRP) {
    // every CTA combines the G partials in the same fixed order: lane q sums
    // the partials q, q + 32, ... (read from L2), then the butterfly tree
    group_barrier(gs, C);
    if (warp == 0) {
      TP t[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        t[k] = (TP)0;
        for (int q = lane; q < C; q += 32)
          t[k] = combine(t[k], (TP)__ldcg(gs.slot + (par * 8 + k) * C + q), op);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t[k] = combine(t[k], __shfl_xor_sync(0xffffffffu, t[k], o), op);
      }
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) bc[k] = (double)t[k];
        post(bc);
      }
    }
  } else if (C > 1) {
    cl.sync();
    if (warp == 0) {
      TP t[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        t[k] = lane < C ? (TP)slot[par * 64 + k * 16 + lane] : (TP)0;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) t[k] = combine(t[k], __shfl_xor_sync(0xffffffffu, t[k], o), op);
      }
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) bc[k] = (double)t[k];
        post(bc);
      }
    }
  }
  __syncthreads();
  par ^= 1;
}

struct NoPost {
  __device__ void operator()(double*) const {}
};

// Packed coordinates and interior flag of node A (the per-node code of the
// kernel) computed from the index, for the global-memory layout: the hot
// passes then issue their stencil loads without first waiting for a load of
// the code.
template <int DIM>
__device__ __forceinline__ unsigned gm_code(const Band& b, int A) {
  const int jk = A / b.N0;
  const int i = A - jk * b.N0;
  const int k = jk / b.N1;
  const int j = jk - k * b.N1;
  const bool in = i > 0 && i < b.N0 - 1 && (DIM < 2 || (j > 0 && j < b.N1 - 1)) &&
                  (DIM <= 2 || (k > 0 && k < b.N2 - 1));
  return (unsigned)i | ((unsigned)j << 11) | ((unsigned)k << 22) | (in ? 0x80000000u : 0u);
}

}  // namespace

// Byte offsets of the per-CTA shared-memory arrays; every array starts on a
// 16-byte boundary.  Used by the kernel's carve-up and the host's sizing.
struct SmemLayout {
  size_t u0, u1, F, r, z, p, q, d, hm, pinv, cs, code, red, slot, bc, total;
};

__host__ __device__ inline SmemLayout smem_layout(int dim, int nmax, int kr, bool coef_smem, int nt) {
  SmemLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = (o + bytes + 15) & ~(size_t)15;
    return at;
  };
  const size_t n8 = (size_t)nmax * 8, nk = (size_t)nmax * kr;
  L.u0 = take(n8); L.u1 = take(n8); L.F = take(n8);
  L.r = take(nk); L.z = take(nk); L.p = take(nk); L.q = take(nk); L.d = take(nk);
  L.hm = take(nk); L.pinv = take(nk);
  L.cs = take(coef_smem ? (size_t)n_offsets(dim) * nk : 0);
  L.code = take((size_t)nmax * 4);
  L.red = take((size_t)4 * 32 * 8);
  L.slot = take((size_t)2 * 4 * 16 * 8);
  L.bc = take(16 * 8);
  L.total = o;
  return L;
}

// The global-memory layout is latency-bound on its streamed couplings: it is
// compiled for two CTAs per SM (64 registers; the Newton and line-search
// phases spill a few words), which doubles the warps in flight on the CG
// passes -- 1.5-1.8x faster on the 3D levels than one CTA with 128 registers.
template <typename KR, int DIM, int NT, int NPT, bool GM, bool MG, bool GRP = false>
__global__ void __launch_bounds__(NT, GM ? 1024 / NT : 1)
solve_cluster_kernel(LevelDesc lv, Physics ph, SolverParams sp, const double* __restrict__ coef64,
                     const KR* __restrict__ coefK, int H, int coef_smem, double* slab,
                     double* t_act, mlmc_sample_info* info, unsigned long long* counters,
                     double* g_u, double* g_F, KR* g_kr, unsigned* g_code, const MGDesc mg,
                     KR* g_mg, int G, unsigned* g_sync, double* g_slot) {
  static_assert(!MG || GM, "the multigrid preconditioner needs the global-memory layout");
  static_assert(!GRP || (GM && !MG), "the group layout is the global-memory layout with Jacobi");
  constexpr int NO = DIM == 3 ? 27 : (DIM == 2 ? 9 : 3);
  constexpr int CTR = DIM == 3 ? 13 : (DIM == 2 ? 4 : 1);
  cg::cluster_group cl = cg::this_cluster();
  Band b;
  __shared__ int s_ticket, s_abort;
  GroupSync gs;
  int s;
  if (GRP) {
    // group layout: sample s = ticket / G, rank = ticket % G in arrival order
    if (threadIdx.x == 0) {
      s_ticket = (int)atomicAdd(g_sync, 1u);
      s_abort = 0;
    }
    __syncthreads();
    b.C = G;
    b.rank = s_ticket % G;
    s = s_ticket / G;
    gs.ctr = g_sync + 32 * (s + 1);
    gs.flag = gs.ctr + 1;
    gs.slot = g_slot + (int64_t)s * 16 * G;
    gs.abort = &s_abort;
    gs.check = sp.grp_check;
  } else {
    b.C = (int)cl.num_blocks();
    b.rank = (int)cl.block_rank();
    s = blockIdx.x / b.C;
  }
  b.N0 = lv.N[0]; b.N1 = lv.N[1]; b.N2 = lv.N[2];
  b.rowlen = DIM == 3 ? b.N0 * b.N1 : b.N0;
  b.nrows = DIM == 3 ? b.N2 : b.N1;
  b.H = H;
  const int N = (int)lv.nodes;
  // Global-memory layout with Jacobi (CYC): the nodes are dealt to the CTAs
  // in chunks of NT, cyclically (CTA r takes chunks r, r + C, ...), so that
  // every CTA gets the same share of boundary nodes -- with contiguous ranges
  // the CTAs that own a whole boundary plane run the slower bounds-checked
  // stencil on every node, and every barrier waits for them.
  constexpr bool CYC = GM && !MG;
  if (GM) {
    // H nodes per CTA, contiguous (multigrid), or every node reachable (CYC)
    b.base = CYC ? 0 : min(b.rank * H, N);
    b.nb = CYC ? N : min(H, N - b.base);
    b.row0 = b.row1 = 0;
    b.nmax = H;
  } else {
    b.row0 = min(b.rank * H, b.nrows);
    b.row1 = min(b.row0 + H, b.nrows);
    b.nb = (b.row1 - b.row0) * b.rowlen;
    b.nmax = H * b.rowlen;
    b.base = b.row0 * b.rowlen;
  }
  const int base = b.base;
  // this thread's nodes a (A = base + a): a_first, a_first + a_step, ... < a_end
  const int a_first = CYC ? b.rank * NT + (int)threadIdx.x : (int)threadIdx.x;
  const int a_step = CYC ? b.C * NT : NT;
  const int a_end = b.nb;
  const int nmax = b.nmax;
  const int N01 = b.N0 * b.N1;
  const int tid = threadIdx.x;

  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(DIM, GM ? 0 : nmax, (int)sizeof(KR), !GM && coef_smem != 0, NT);
  double* ubuf0 = GM ? g_u + (int64_t)s * 2 * N + base : (double*)(smem + L.u0);
  double* ubuf1 = GM ? g_u + (int64_t)s * 2 * N + N + base : (double*)(smem + L.u1);
  double* F = GM ? g_F + (int64_t)s * N + base : (double*)(smem + L.F);
  KR* const kr0 = GM ? g_kr + (int64_t)s * 7 * N + base : nullptr;
  KR* r = GM ? kr0 : (KR*)(smem + L.r);
  KR* z = GM ? kr0 + N : (KR*)(smem + L.z);
  KR* p = GM ? kr0 + 2 * N : (KR*)(smem + L.p);
  KR* q = GM ? kr0 + 3 * N : (KR*)(smem + L.q);
  KR* d = GM ? kr0 + 4 * N : (KR*)(smem + L.d);
  KR* hm = GM ? kr0 + 5 * N : (KR*)(smem + L.hm);
  KR* pinv = GM ? kr0 + 6 * N : (KR*)(smem + L.pinv);
  KR* cs = (KR*)(smem + L.cs);                             // couplings [NO][nmax] if coef_smem
  double* red = (double*)(smem + L.red);
  double* slot = (double*)(smem + L.slot);
  double* bc = (double*)(smem + L.bc);
  KR* const bck = (KR*)(bc + 8);   // KR copies of broadcast scalars
  int par = 0;

  // 3D global-memory sweeps read the couplings stored once per symmetric pair
  constexpr bool SYM = GM && !MG && DIM == 3;
  constexpr int NOS = SYM ? NO - CTR : NO;
  const double* c64 = coef64 + (int64_t)s * NOS * N;
  const KR* cKg = coefK + (int64_t)s * NOS * N;
  double* ta = t_act + (int64_t)s * N;
  double* sl = slab ? slab + (int64_t)s * (lv.m + 1) * N : nullptr;
  const double dt = lv.dt, inv_dt = 1.0 / lv.dt;

  // Per node: packed coordinates i | j << 11 | k << 22 and, in bit 31, whether
  // every neighbour lies inside the domain and inside this band (then the
  // stencil uses constant local offsets).
  unsigned* code = GM ? g_code + (int64_t)s * N + base : (unsigned*)(smem + L.code);
  for (int a = a_first; a < a_end; a += a_step) {
    int i, j, k, row;
    if (GM) {
      const int A = base + a;
      i = A % b.N0;
      j = (A / b.N0) % b.N1;
      k = A / N01;
      row = DIM == 3 ? k : j;
    } else {
      const int lr = a / b.rowlen, inrow = a - lr * b.rowlen;
      row = b.row0 + lr;
      if (DIM == 3) { k = row; j = inrow / b.N0; i = inrow - j * b.N0; }
      else { k = 0; j = row; i = inrow; }
    }
    bool in = i > 0 && i < b.N0 - 1 && (DIM < 2 || (j > 0 && j < b.N1 - 1)) &&
              (DIM <= 2 || (k > 0 && k < b.N2 - 1));
    bool fast = in && (GM || (row > b.row0 && row < b.row1 - 1));
    code[a] = (unsigned)i | ((unsigned)j << 11) | ((unsigned)k << 22) | (fast ? 0x80000000u : 0u);
  }
#define CI(c) ((int)((c) & 2047u))
#define CJ(c) ((int)(((c) >> 11) & 2047u))
#define CK_(c) ((int)(((c) >> 22) & 511u))
#define CFAST(c) (((c) & 0x80000000u) != 0u)

  if (!GRP) cl.sync();   // every CTA of the cluster is resident before any DSMEM access

  KR* const mgb = MG ? g_mg + (int64_t)s * mg.per_sample : nullptr;
  if (MG) gmg::build<NT, DIM, KR>(mg, mgb, coef64 + (int64_t)s * NO * N, cl, b.C, b.rank);

  if (!GM && coef_smem)
    for (int o = 0; o < NO; ++o)
      for (int a = a_first; a < a_end; a += a_step) cs[o * nmax + a] = cKg[(int64_t)o * N + base + a];
  double sc[3];
  for (int dd = 0; dd < 3; ++dd) sc[dd] = ph.stim_ps ? ph.stim_ps[3 * s + dd] : ph.stim_c[dd];
  for (int a = a_first; a < a_end; a += a_step) {
    const unsigned c = code[a];
    const int A = base + a;
    double x[3] = {CI(c) * lv.h[0], CJ(c) * lv.h[1], CK_(c) * lv.h[2]};
    double r2 = 0.0;
    for (int dd = 0; dd < DIM; ++dd) r2 += (x[dd] - sc[dd]) * (x[dd] - sc[dd]);
    double v = ph.stim_kind == 0 && r2 < ph.stim_r2 ? 1.0 : 0.0;
    ubuf0[a] = v;
    ta[A] = v >= 0.5 ? 0.0 : -1.0;
    if (sl) sl[A] = v;
  }
  const View<KR> pv = make_view<GM>(cl, b, p);
  const View<KR> zview = make_view<GM>(cl, b, z);
  const View<KR> dv = make_view<GM>(cl, b, d);
  const View<double> uv0 = make_view<GM>(cl, b, ubuf0);
  const View<double> uv1 = make_view<GM>(cl, b, ubuf1);
  const double rtol2 = sp.lin_rtol * sp.lin_rtol;

  int status = MLMC_OK, failed_step = 0;
  int newton_total = 0, cg_total = 0, trunc_total = 0, halvings = 0, max_newton = 0;
  for (int step = 1; step <= lv.m; ++step) {
    double* u = (step & 1) ? ubuf1 : ubuf0;
    const double* up = (step & 1) ? ubuf0 : ubuf1;
    const View<double>& uv = (step & 1) ? uv1 : uv0;
    const View<double>& upv = (step & 1) ? uv0 : uv1;
    // explicit part of the residual: (1-theta)/theta times the (theta-scaled)
    // stencil of u_{k-1} (Crank-Nicolson), and the applied current's step average
    const double c_up = (1.0 - ph.theta) / ph.theta;
    const double src_scale = stim_step_scale(ph, step, dt);
    // start: u_{k-1}, or on levels with a unique root (no continuation) the
    // linear extrapolation 2 u_{k-1} - u_{k-2} (the buffer u still holds
    // u_{k-2}), which the root does not depend on
    const bool extrap = !sp.flow && step >= 2;
    for (int a = a_first; a < a_end; a += a_step) u[a] = extrap ? 2.0 * up[a] - u[a] : up[a];
    sync_all<GRP>(cl, b.C, gs);
    // On levels whose steps have several roots (sp.flow) the step follows the
    // gradient-flow continuation (see SolverParams).
    double tau = sp.tau0, sw = FLOW_NEWTON;
    bool newton_phase = false;
    bool conv = false, lin_fail = false;
    int it;
    for (it = 1; it <= sp.newton_max; ++it) {
      if (GRP && s_abort) break;   // a group wait ran out: stop
      // pseudo-step of the continuation (shift = M/t on the Hessian diagonal),
      // or a Newton step (shift 0)
      const double t = tau;
      const double shift = sp.flow && !newton_phase ? 1.0 / t : 0.0;
      // residual, Hessian diagonal and the CG start r = -F, z = P^-1 r, p = z, d = 0
      // FP32 CG on grids with a tiny lumped mass per time step (sp.cg_scale,
      // the fine 3D levels): the right-hand side is scaled by a power of two
      // sigma with ||F||_2 sigma in [1, 2), and d by 1/sigma after the solve.
      // Both are exact, so this changes nothing except that the CG's products
      // stay in FP32's normal range: on the 256 x 256 x 64 level (lumped mass
      // ~ h^3) the late Newton residuals are ~1e-18 and the CG's r.z fell below
      // 1e-38.  One FP64 reduction gives sum F^2 (for sigma) and sum F^2 /
      // |H_ii| (the CG's first r.z, = sigma^-2 r.z), so the scaling costs one
      // local pass and a barrier per Newton iteration.
      const bool SCALE = sizeof(KR) == 4 && sp.cg_scale != 0;
      double f2_loc = 0.0, f2p_loc = 0.0;
      KR rz_loc = 0;
      for (int a = a_first; a < a_end; a += a_step) {
        const unsigned c = GM ? gm_code<DIM>(b, base + a) : code[a];
        const int A = base + a;
        auto c64A = [=](int o) { return coupling<SYM, DIM>(c64, o, N, A, b.N0, N01); };
        double ku = stencil_node<DIM, GM, double>(b, u, uv, a, c, N01, c64A, sp.pred_stencil);
        if (c_up != 0.0)
          ku += c_up * (stencil_node<DIM, GM, double>(b, up, upv, a, c, N01, c64A, sp.pred_stencil));
        const double mA = lumped_mass(lv, CI(c), CJ(c), CK_(c)), uA = u[a];
        double f = ku + mA * inv_dt * (uA - up[a]) - mA * rxn(ph, uA);
        if (src_scale != 0.0) f -= mA * src_scale * stim_shape(ph, lv, sc, CI(c), CJ(c), CK_(c));
        F[a] = f;
        // Hessian diagonal and Jacobi inverse in the CG's precision (the CG is
        // the only user); no FP64 division on the per-node path
        const KR uK = (KR)uA, mK = (KR)mA;
        const KR rdK = (KR)ph.c * ((KR)(-3.0) * uK * uK + (KR)(2.0 * (1.0 + ph.a)) * uK - (KR)ph.a);
        const KR hmA = mK * ((KR)(inv_dt + shift) - rdK);
        hm[a] = hmA;
        d[a] = (KR)0;
        const KR pvv = MG ? (KR)1 / (fabs(hmA) + mgb[mg.l[0].ks + A])   // l1-Jacobi (V-cycle smoother)
                          : (KR)1 / fabs(hmA + (KR)c64[(int64_t)(SYM ? 0 : CTR) * N + A]);
        pinv[a] = pvv;
        if (SCALE) {
          f2_loc += f * f;
          f2p_loc += f * f * (double)pvv;
        } else {
          const KR rv = (KR)(-f);
          r[a] = rv;
          if (!MG) {
            const KR zv = pvv * rv;
            z[a] = zv; p[a] = zv;
            rz_loc += rv * zv;
          }
        }
      }
      double sigma = 1.0, rz_scaled = 0.0;
      if (SCALE) {
        double v2[2] = {f2_loc, f2p_loc};
        cluster_reduce<NT, double, 2, GRP>(v2, 0, red, slot, bc, par, cl, b.C, b.rank, gs, NoPost());
        if (bc[0] > 0.0) sigma = ldexp(1.0, -ilogb(sqrt(bc[0])));
        rz_scaled = bc[1] * sigma * sigma;
        for (int a = a_first; a < a_end; a += a_step) {
          const KR rv = (KR)(-F[a] * sigma);
          r[a] = rv;
          if (!MG) {
            const KR zv = pinv[a] * rv;
            z[a] = zv; p[a] = zv;
          }
        }
        if (!MG) sync_all<GRP>(cl, b.C, gs);   // p is read across the cluster next
      }
      if (MG) {
        sync_all<GRP>(cl, b.C, gs);
        gmg::newton_setup<NT, DIM, KR>(mg, mgb, hm - base, cl, b.C, b.rank);
        gmg::vcycle<NT, DIM, KR>(mg, mgb, cKg, hm - base, pinv - base, r - base, z - base, cl, b.C,
                                 b.rank);
        for (int a = a_first; a < a_end; a += a_step) {
          const KR zv = z[a];
          p[a] = zv;
          rz_loc += r[a] * zv;
        }
      }
      if (MG || !SCALE) {
        KR v1[1] = {rz_loc};
        cluster_reduce<NT, KR, 1, GRP>(v1, 0, red, slot, bc, par, cl, b.C, b.rank, gs, NoPost());
      }
      double rz = MG || !SCALE ? bc[0] : rz_scaled;
      const double rz_stop = rtol2 * rz;
      int cgi = 0;
      bool truncated = false;
      if (rz > 0.0) {
        bool ok = false;
        // From the second iteration on, the search direction p = z + beta p
        // and q = H p are formed in the same pass as the stencil, from
        // H p = H z + beta q (the stencil is applied to z, which the last
        // reduction's cluster barrier published): no separate pass and
        // cluster barrier for the new p.
        KR beta_prev = 0;
        for (cgi = 1; cgi <= sp.lin_max; ++cgi) {
          KR pq_loc = 0;
          const bool first = cgi == 1;
          const KR* sv = first ? p : z;               // the vector the stencil reads
          const View<KR>& svv = first ? pv : zview;
          for (int a = a_first; a < a_end; a += a_step) {
            const unsigned c = GM ? gm_code<DIM>(b, base + a) : code[a];
            const int A = base + a;
            KR hs;
            if (!GM && coef_smem) {
              auto cf = [=](int o) { return cs[o * nmax + a]; };
              hs = stencil_node<DIM, GM, KR>(b, sv, svv, a, c, N01, cf, sp.pred_stencil);
            } else {
              auto cf = [=](int o) { return coupling<SYM, DIM>(cKg, o, N, A, b.N0, N01); };
              hs = stencil_node<DIM, GM, KR>(b, sv, svv, a, c, N01, cf, sp.pred_stencil);
            }
            const KR sa = sv[a];
            KR pa, qv;
            if (first) {
              pa = sa;
              qv = hs + hm[a] * sa;
            } else {
              pa = sa + beta_prev * p[a];
              qv = (hs + hm[a] * sa) + beta_prev * q[a];
              p[a] = pa;
            }
            q[a] = qv;
            pq_loc += pa * qv;
          }
          const double rzc = rz;
          {
            KR v1[1] = {pq_loc};
            cluster_reduce<NT, KR, 1, GRP>(v1, 0, red, slot, bc, par, cl, b.C, b.rank, gs, [=](double* o) {
              o[1] = o[0] > 0.0 ? (double)((KR)rzc / (KR)o[0]) : 0.0;
              bck[0] = (KR)o[1];
              bck[1] = o[0] <= 0.0 ? (KR)1 : (KR)0;
            });
          }
          if (GRP && s_abort) break;
          // the scalars every thread needs, read in KR: no FP64 operation per
          // thread and iteration (FP64 runs at 1/64 of the FP32 rate here)
          if (bck[1] != (KR)0) {
            truncated = true;
            if (cgi == 1)
              for (int a = a_first; a < a_end; a += a_step) d[a] = z[a];
            ok = true;
            break;
          }
          const KR alpha = bck[0];
          KR rzn_loc = 0;
          if (MG) {
            for (int a = a_first; a < a_end; a += a_step) {
              d[a] += alpha * p[a];
              r[a] = r[a] - alpha * q[a];
            }
            sync_all<GRP>(cl, b.C, gs);
            gmg::vcycle<NT, DIM, KR>(mg, mgb, cKg, hm - base, pinv - base, r - base, z - base, cl,
                                     b.C, b.rank);
            for (int a = a_first; a < a_end; a += a_step) rzn_loc += r[a] * z[a];
          } else {
            for (int a = a_first; a < a_end; a += a_step) {
              d[a] += alpha * p[a];
              const KR rv = r[a] - alpha * q[a];
              const KR zv = pinv[a] * rv;
              r[a] = rv;
              z[a] = zv;
              rzn_loc += rv * zv;
            }
          }
          {
            KR v1[1] = {rzn_loc};
            cluster_reduce<NT, KR, 1, GRP>(v1, 0, red, slot, bc, par, cl, b.C, b.rank, gs, [=](double* o) {
              o[1] = (double)((KR)o[0] / (KR)rzc);
              o[2] = o[0] <= rz_stop ? 1.0 : 0.0;
              bck[2] = (KR)o[1];
              bck[3] = (KR)o[2];
            });
          }
          if (GRP && s_abort) break;
          if (bck[3] != (KR)0) { ok = true; break; }
          beta_prev = bck[2];
          rz = bc[0];
        }
        if (!ok) { lin_fail = true; cgi = sp.lin_max; }
      }
      cg_total += cgi;
      trunc_total += truncated ? 1 : 0;
      if (lin_fail) break;
      if (SCALE && sigma != 1.0) {
        const KR inv_sigma = (KR)(1.0 / sigma);   // a power of two: exact
        for (int a = a_first; a < a_end; a += a_step) d[a] *= inv_sigma;
      }
      KR dm_loc = 0;
      for (int a = a_first; a < a_end; a += a_step) dm_loc = fmax(dm_loc, fabs(d[a]));   // exact in KR
      {
        KR v1[1] = {dm_loc};
        cluster_reduce<NT, KR, 1, GRP>(v1, 1, red, slot, bc, par, cl, b.C, b.rank, gs, NoPost());
      }
      const double dmax = bc[0];
      if (sp.flow) {
        bool accept;
        if (newton_phase) {
          accept = !(truncated || dmax > 10.0 * sw);
          if (!accept) { newton_phase = false; sw *= 0.1; ++halvings; }
        } else if (truncated && t > FLOW_TMIN) {
          accept = false;              // M/t + H not positive definite
          tau = 0.25 * t;
          ++halvings;
        } else {
          accept = true;
        }
        if (!accept) continue;       // the state is unchanged; retry
        if (!newton_phase && dmax > FLOW_MOVE && t > FLOW_TMIN) {
          // the step would move a node by more than FLOW_MOVE: take it
          // shortened to that move (a positive multiple keeps its sign along
          // every eigenvector of M/t + H); the next pseudo-step is shorter
          const double sc = FLOW_MOVE / dmax;
          for (int a = a_first; a < a_end; a += a_step) u[a] += sc * (double)d[a];
          sync_all<GRP>(cl, b.C, gs);
          tau = t * 0.9 * sc;
          ++halvings;
          continue;
        }
        for (int a = a_first; a < a_end; a += a_step) u[a] += (double)d[a];
        sync_all<GRP>(cl, b.C, gs);
        if (dmax <= sp.newton_tol) { conv = true; break; }
        if (!newton_phase) {
          if (dmax <= sw) newton_phase = true;
          tau = fmin(t * fmin(2.0, 0.9 * FLOW_MOVE / dmax), FLOW_TMAX);   // towards the move limit
        }
        continue;
      }
      double alpha = 1.0;
      if (dmax > sp.newton_tol && dmax > sp.ls_full_step) {
        // The step energy is a quartic polynomial in the step length (R is a
        // quartic), so for every trial length al
        //   E(u + al d) - E(u) = al g.d + al^2 d.Hd / 2 - al^3 P3 - al^4 P4,
        //   P3 = sum_i m_i r2(u_i) d_i^3 / 6,  P4 = sum_i m_i r3 d_i^4 / 24,
        // with r2 = r'' = c(2(1+a) - 6u) and r3 = r''' = -6c; one pass over the
        // nodes gives the four sums and thread 0 runs every Armijo test.
        // The sums run in the inner solve's precision KR (FP32 on mixed
        // levels): they only choose the step length, and the root that the
        // Newton iteration converges to does not depend on it.  d.Hd takes
        // the Hessian's diagonal mass term hm = m (1/dt - r'(u)) of this
        // iteration (the shift is 0 outside the continuation).
        KR v4[4] = {0, 0, 0, 0};
        for (int a = a_first; a < a_end; a += a_step) {
          const unsigned c = GM ? gm_code<DIM>(b, base + a) : code[a];
          const int A = base + a;
          KR kd;
          if (!GM && coef_smem) {
            auto cf = [=](int o) { return cs[o * nmax + a]; };
            kd = stencil_node<DIM, GM, KR>(b, d, dv, a, c, N01, cf, sp.pred_stencil);
          } else {
            auto cf = [=](int o) { return coupling<SYM, DIM>(cKg, o, N, A, b.N0, N01); };
            kd = stencil_node<DIM, GM, KR>(b, d, dv, a, c, N01, cf, sp.pred_stencil);
          }
          const KR mK = (KR)lumped_mass(lv, CI(c), CJ(c), CK_(c));
          const KR uK = (KR)u[a], da = d[a], d2 = da * da;
          const KR r2 = (KR)ph.c * ((KR)(2.0 * (1.0 + ph.a)) - (KR)6.0 * uK);
          v4[0] += (KR)F[a] * da;
          v4[1] += hm[a] * d2 + da * kd;
          v4[2] += mK * r2 * d2 * da;
          v4[3] += mK * d2 * d2;
        }
        const double alpha0 = alpha, cc = ph.c;   // alpha0 = 1
        cluster_reduce<NT, KR, 4, GRP>(v4, 0, red, slot, bc, par, cl, b.C, b.rank, gs,
                                      [=](double* o) {
                                        const double gd = o[0], dHd = o[1];
                                        const double P3 = o[2] / 6.0, P4 = -6.0 * cc * o[3] / 24.0;
                                        double al = alpha0;
                                        int h = 0;
                                        for (; h < 40; ++h) {
                                          const double dE = al * gd + 0.5 * al * al * dHd -
                                                            al * al * al * P3 - al * al * al * al * P4;
                                          if (dE <= 1e-4 * al * gd) break;
                                          al *= 0.5;
                                        }
                                        o[4] = al;
                                        o[5] = (double)h;
                                      });
        alpha = bc[4];
        halvings += (int)bc[5];
      }
      for (int a = a_first; a < a_end; a += a_step) u[a] += alpha * (double)d[a];
      sync_all<GRP>(cl, b.C, gs);
      if (dmax <= sp.newton_tol) { conv = true; break; }
    }
    int used = it > sp.newton_max ? sp.newton_max : it;
    newton_total += used;
    max_newton = used > max_newton ? used : max_newton;
    if (!conv) {
      status = GRP && s_abort ? MLMC_ERR_TIMEOUT : MLMC_ERR_NOT_CONVERGED;
      failed_step = step;
      break;
    }
    for (int a = a_first; a < a_end; a += a_step) {
      const int A = base + a;
      if (ta[A] < 0.0 && u[a] >= 0.5) {
        double uo = up[a];
        ta[A] = (double)(step - 1) * dt + dt * (0.5 - uo) / (u[a] - uo);
      }
      if (sl) sl[(int64_t)step * N + A] = u[a];
    }
  }
#undef CI
#undef CJ
#undef CK_
#undef CFAST
  {
    // the quantity of interest: activation times (T where never reached), or
    // the final state u(T) (in the buffer of step m)
    const double* ufin = (lv.m & 1) ? ubuf1 : ubuf0;
    for (int a = a_first; a < a_end; a += a_step) {
      if (ph.qoi == 1) ta[base + a] = ufin[a];
      else if (ta[base + a] < 0.0) ta[base + a] = lv.T;
    }
  }
  if (b.rank == 0 && tid == 0) {
    if (counters) {
      if (status != MLMC_OK) atomicAdd(counters, 1ull);
      atomicAdd(counters + 1, (unsigned long long)cg_total * (unsigned long long)N);
      atomicAdd(counters + 2, (unsigned long long)newton_total * (unsigned long long)N);
      atomicAdd(counters + 3, (unsigned long long)trunc_total);
      atomicAdd(counters + 4, (unsigned long long)halvings);
      if (sizeof(KR) == 8) atomicAdd(counters + 5, (unsigned long long)cg_total * (unsigned long long)N);
    }
    if (info) {
      mlmc_sample_info o;
      o.status = status; o.failed_step = failed_step; o.newton_iters = newton_total;
      o.cg_iters = cg_total; o.truncations = trunc_total; o.halvings = halvings;
      o.max_newton = max_newton; o.pad = 0;
      info[s] = o;
    }
  }
  if (!GRP) cl.sync();   // no CTA leaves while a neighbour may still read its shared memory
}

template <typename KR, int DIM, bool GM, bool MG = false, bool GRP = false, int NT = 512>
inline cudaError_t set_attrs(const ClusterPlan& pl) {
  auto kern = solve_cluster_kernel<KR, DIM, NT, 5, GM, MG, GRP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e == cudaSuccess && !GRP && pl.C > 8)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// Launch configuration: n clusters of C CTAs of pl.nt threads, or (group
// layout, pl.G > 0) a plain grid of n groups of G CTAs.
inline cudaLaunchConfig_t launch_cfg(const ClusterPlan& pl, int n, cudaStream_t st,
                                     cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * pl.C));
  cfg.blockDim = dim3((unsigned)pl.nt);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pl.G > 0 ? 1 : pl.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = pl.G > 0 ? 0 : 1;
  return cfg;
}

template <typename KR, int DIM, bool GM, bool MG, bool GRP = false, int NT = 512>
inline cudaError_t launch_one(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                              const ClusterPlan& pl, int n, const double* coef64, const KR* coefK,
                              double* slab, double* t_act, mlmc_sample_info* info,
                              unsigned long long* counters, const ClusterGlobal& g,
                              const MGDesc& mg, cudaStream_t st) {
  if (pl.nt != NT) return cudaErrorInvalidValue;
  cudaError_t e = set_attrs<KR, DIM, GM, MG, GRP, NT>(pl);
  if (e != cudaSuccess) return e;
  if (GRP) {
    // tickets and barrier counters start from zero in every launch
    e = cudaMemsetAsync(g.gsync, 0, group_sync_bytes(n), st);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = launch_cfg(pl, n, st, at);
  return cudaLaunchKernelEx(&cfg, solve_cluster_kernel<KR, DIM, NT, 5, GM, MG, GRP>, lv, ph, sp,
                            coef64, coefK, pl.H, pl.coef_smem ? 1 : 0, slab, t_act, info, counters,
                            g.u, g.F, (KR*)g.kr, g.code, mg, (KR*)g.mg, GRP ? pl.G : 0, g.gsync,
                            g.gslot);
}


}  // namespace mlmc
