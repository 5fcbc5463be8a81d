// One-level space-time restricted additive Schwarz preconditioner (Sec. 3.2)
// with ILU(0) subdomain solves, all subdomains in one launch.
//
// Subdomains.  The node range of each axis and the level range 0..M are cut
// into nsub parts (part k of n holds floor(n/p) + (k < n mod p)); a box is the
// product of one part per axis (owned set), extended by `overlap` on every
// side and trimmed to the domain (extended set, Fig. 1).  The subdomain
// matrix M_ij is the principal submatrix of F_h on the extended set, i.e. the
// discretisation with homogeneous Dirichlet data on every cut face in space
// and time (Eq. 10-12).
//
// Storage.  A row of F_h is described by its row type (C, G or f) and a fixed
// list of slots (level offset dt, spatial offset, column component) -- the
// structural stencil of that block row, ordered as the columns are ordered
// (time slowest, then z, y, x, then component).  Every point of a box stores
// 108 + 56 + 162 = 326 slot values, no column indices; slots whose column is
// outside the box hold 0, which is the same as leaving them out of the
// pattern.
//
// Layout in HBM.  The points of each wavefront are cut into chunks of at most
// CH points (56 in FP32, 28 in FP64).  A chunk's values form one contiguous
// block [slot rank][point of the chunk] with a row stride cp >= the chunk's
// point count chosen so that the shared-memory reads of the solve are free of
// bank conflicts; the L-slots of the three rows come first (175 ranks), then
// the diagonal and U-slots (151 ranks).  The forward sweep therefore streams
// one contiguous L block per chunk and the backward sweep one U block.
//
// Ordering and parallelism.  Points are processed in the natural
// (lexicographic) order of the box; with this stencil every lower-triangular
// dependency of point (x, y, z, t) lies on a wavefront w' < w where
// w = x + 2y + 4z + 8t, so all points of one wavefront are independent.  Within
// a point the rows go C, G, f.  One CTA owns one box and steps through its
// wavefronts with a barrier between them.
//
// ILU(0) (IKJ form, on the structural pattern):
//   for each row i in order, for each k < i in pattern(i) ascending:
//     a_ik /= u_kk;  a_ij -= a_ik u_kj  for j > k in pattern(i) and pattern(k).
// The (row slot, column slot) pairs of the inner update are fixed per row
// type and written out as straight-line code (ilu_rows.inc).  The diagonal
// slot of a factored row stores 1/u_kk, so both the factorisation and the
// backward sweep multiply instead of divide.
//
// Solve.  One CTA per box runs a two-stage pipeline over its chunks: thread 0
// issues a TMA bulk copy (cp.async.bulk, completion on an mbarrier) of the
// next chunk's L (or U) block into one of two shared-memory buffers while the
// CTA computes the current chunk from the other.  The local vector of each box
// has a ghost layer of zeros one point wide in every direction, so the
// triangular sweeps need no bounds tests: a slot whose column leaves the box
// reads 0 and has factor value 0.  Small boxes keep the local vector in shared
// memory as well.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "ras.cuh"

namespace {

// ---------------------------------------------------------------------------
// slot tables (host-built, copied to constant memory)
// ---------------------------------------------------------------------------
struct SlotTables {
  // per slot (0..325): packed offsets
  int8_t dt[kSlots], dz[kSlots], dy[kSlots], dx[kSlots], comp[kSlots];
  int base[3], count[3], diag[3];       // diag = absolute slot index of the diagonal
};

SlotTables build_tables() {
  SlotTables T;
  int s = 0;
  for (int c = 0; c < 3; ++c) {
    T.base[c] = s;
    const int dt_lo = (c == 1) ? 0 : -1;
    const int dt_hi = (c == 0) ? 0 : 1;
    for (int dt = dt_lo; dt <= dt_hi; ++dt)
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx)
            for (int cc = 0; cc < 3; ++cc) {
              bool use;
              if (c == 0) use = (cc == 0 || cc == 2);
              else if (c == 1) use = (cc == 1) || (cc == 0 && dx == 0 && dy == 0 && dz == 0);
              else use = (cc == 1 || cc == 2);
              if (!use) continue;
              T.dt[s] = (int8_t)dt; T.dz[s] = (int8_t)dz; T.dy[s] = (int8_t)dy; T.dx[s] = (int8_t)dx;
              T.comp[s] = (int8_t)cc;
              if (dt == 0 && dz == 0 && dy == 0 && dx == 0 && cc == c) T.diag[c] = s;
              ++s;
            }
    T.count[c] = s - T.base[c];
  }
  return T;
}

const SlotTables& tables() {
  static const SlotTables T = build_tables();
  return T;
}

// Checksum of the slot list and chunk block rank of every slot, as the
// generated factorisation code (factor32.cu, factor64.cu) assumes them.
#include "ilu_slots.inc"

// Slot ranges of the three row types (checked against the tables on the host).
constexpr int kCBase = 0, kCDiag = 80, kCEnd = 108;
constexpr int kGBase = 108, kGDiag = 122, kGEnd = 164;
constexpr int kFBase = 164, kFDiag = 245, kFEnd = 326;
// span of a box's unit row: kSlots rounded up to whole 16-byte units in FP32 and FP64
constexpr int kUnitRowSpan = (kSlots + 3) / 4 * 4;
constexpr int kLRanks = 175;        // L-slots of the three rows
constexpr int kURanks = 151;        // diagonals and U-slots of the three rows

// rank of slot s in a chunk block: L-slots of C, G, f, then diag+U of C, G, f
int slot_rank(int s) {
  if (s < kCDiag) return s;
  if (s >= kGBase && s < kGDiag) return 80 + (s - kGBase);
  if (s >= kFBase && s < kFDiag) return 94 + (s - kFBase);
  if (s >= kCDiag && s < kCEnd) return kLRanks + (s - kCDiag);
  if (s >= kGDiag && s < kGEnd) return kLRanks + 28 + (s - kGDiag);
  return kLRanks + 70 + (s - kFDiag);
}

// Chunk configurations of the subdomain solve, per stored type S: candidate
// chunk sizes (points) and the row-stride rule cp = R (mod Q) of a chunk
// block.  In a step the 4 lanes of a point take the stencil neighbours
// q = lane + 4 i; the factor entries of neighbour q in the C and f rows sit
// in block rows a + 2q (+1), so the 4 lanes of a point read rows 2 apart and
// the 8 points of a warp read 8 consecutive columns: with 2 cp = 8 (mod 32)
// 4-byte words the 32 reads of a warp fall in 32 different banks (for 8-byte
// values every half warp does; for 2-byte values, two per word).  cp is also
// a multiple of 16 bytes' worth of values over the 175 and 151 block rows,
// so every bulk copy starts and ends on 16-byte boundaries.
template <typename S>
struct ChunkCfg;
// The chunk sizes are strides the rule allows, so a full chunk carries no
// padding columns.
template <>
struct ChunkCfg<float> {
  static constexpr int CH = 52, CH2 = 36, CH3 = 20;
  static constexpr int Q = 16, R = 4;                  // cp = 4 (mod 16)
};
template <>
struct ChunkCfg<double> {
  static constexpr int CH = 34, CH2 = 26, CH3 = 18;
  static constexpr int Q = 8, R = 2;                   // cp = 2 (mod 8)
};
template <>
struct ChunkCfg<__nv_bfloat16> {                      // FP32 factors stored as BF16
  static constexpr int CH = 72, CH2 = 40, CH3 = 8;
  static constexpr int Q = 32, R = 8;                  // cp = 8 (mod 32): two values per bank word
};
constexpr int kLanes = 4;   // lanes per point of the subdomain solve
// arithmetic type of the solve for a storage type (BF16 factors: FP32)
template <typename S>
struct SolveArith {
  using type = S;
};
template <>
struct SolveArith<__nv_bfloat16> {
  using type = float;
};
template <typename T, typename S>
__device__ __forceinline__ T arith(S v) {
  return static_cast<T>(v);
}
template <>
__device__ __forceinline__ float arith<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename S>
int chunk_stride(int n) {
  const int Q = ChunkCfg<S>::Q, R = ChunkCfg<S>::R;
  return n <= R ? R : R + ((n - R + Q - 1) / Q) * Q;
}
template <typename S>
__host__ __device__ constexpr int chunk_stride_dev(int n) {
  return n <= ChunkCfg<S>::R ? ChunkCfg<S>::R
                             : ChunkCfg<S>::R + ((n - ChunkCfg<S>::R + ChunkCfg<S>::Q - 1) / ChunkCfg<S>::Q) *
                                                    ChunkCfg<S>::Q;
}
static_assert(chunk_stride_dev<float>(ChunkCfg<float>::CH) == ChunkCfg<float>::CH, "full FP32 chunk unpadded");
static_assert(chunk_stride_dev<double>(ChunkCfg<double>::CH) == ChunkCfg<double>::CH, "full FP64 chunk unpadded");
static_assert(chunk_stride_dev<__nv_bfloat16>(ChunkCfg<__nv_bfloat16>::CH) == ChunkCfg<__nv_bfloat16>::CH,
              "full BF16 chunk unpadded");
int chunk_stride_of(int prec, int n) {
  if (prec == 64) return chunk_stride<double>(n);
  if (prec == 16) return chunk_stride<__nv_bfloat16>(n);
  return chunk_stride<float>(n);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on phase `parity` of an mbarrier: gives up after limit_ns
// nanoseconds of polling, records status 2 in *failed and returns false.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s: a block copy takes microseconds
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* failed,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  // the timer is read only every 64 polls, so a copy that lands within the
  // first polls is seen without the timer's latency
  unsigned long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u) {
      const unsigned long long t = global_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > limit_ns) {
        atomicExch(failed, 2);
        return false;
      }
    }
  }
}

// Self-test of the bounded wait (ras_selftest_wait): one thread initialises an
// mbarrier that expects one arrival, which nothing makes, and waits on it for
// limit_ns; the wait gives up, sets *status = 2 and the kernel returns.  No
// copy is issued, so nothing is in flight when the CTA exits.
__global__ void wait_selftest(int* status, unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_fence_init();
  mbar_wait(&bar, 0u, status, limit_ns);
}

// ---------------------------------------------------------------------------
// Subdomain solve z = sum_boxes (R^0)^T M^{-1} R^delta r: one CTA per box,
// 4 lanes per point, one chunk of points per step.
//
// The box's padded local vector holds 4 values per point (C, G, f and a zero),
// so one 16-byte load fetches a neighbour's three unknowns.  Every L-slot of
// the three rows of a point reads one of 40 earlier stencil neighbours (27 at
// level n-1, 13 earlier ones at level n) and every U-slot one of 40 later
// ones (13 at level n, 27 at n+1), besides the point itself.  Lane l takes
// the neighbours q = l + 4 i (i < 10) of both sweeps; it loads their values
// once and forms its parts of the C, G and f row sums from the block rows of
// those slots, which are affine in q (rows counted within the L or U block):
//   forward  C row: 2q + c (c: C, f)   G row: 80 + q - 27 (q >= 27)   f row: 94 + 2q + c (c: G, f)
//   backward C row: 2 + 2q + c (q < 13)   f row: 71 + 2q + c
//            G row: 29 + q (q < 13), 42 + d + (d >= 13) with d = q - 13; the C entry at
//            (n+1, same node), q = 26, in row 55
// and a shuffle reduction over the 4 lanes closes each sum.
// ---------------------------------------------------------------------------
constexpr size_t kSmemLimit = 227 * 1024;          // dynamic shared memory of one CTA
constexpr int kSolveHeader = 2048;   // from byte 1536: the mbarriers and the abort word
constexpr int kMaxStages = 4;        // buffers of the subdomain solve's copy ring
constexpr int kNbr = 40;             // earlier (and later) stencil neighbours of a point
constexpr int kNbrPerLane = kNbr / kLanes;
constexpr int kVecWidth = 4;         // values per point in the local vectors

// the three unknowns of a local-vector point (4 values, 16- or 32-byte aligned)
__device__ __forceinline__ void ld3(const float* p, float& a, float& b, float& c) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = v.x;
  b = v.y;
  c = v.z;
}
__device__ __forceinline__ void ld3(const double* p, double& a, double& b, double& c) {
  const double2 v0 = *reinterpret_cast<const double2*>(p);
  a = v0.x;
  b = v0.y;
  c = p[2];
}
__device__ __forceinline__ void st3(float* p, float a, float b, float c) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, 0.f);
}
__device__ __forceinline__ void st3(double* p, double a, double b, double c) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
  *reinterpret_cast<double2*>(p + 2) = make_double2(c, 0.0);
}

template <typename T>
__device__ __forceinline__ T lane_sum(T v) {
#pragma unroll
  for (int o = 1; o < kLanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// S: type of the stored factor values; T: arithmetic and local-vector type
// threads of a CTA: the lanes of the largest chunk, in whole warps
template <typename S>
constexpr int solve_threads_max() {
  return (ChunkCfg<S>::CH * kLanes + 31) / 32 * 32;
}

// Neighbour q of a point whose wavefront is one away from the point's (w - 1
// in the forward sweep, w + 1 in the backward one): with the wavefront weights
// (1, 2, 4, 8) these are, forward (level n-1: d = q; level n: d = q - 27),
// (1, 1, 1) at n-1 and (1, 1, -1), (1, -1, 0), (-1, 0, 0) at n, and backward
// (level n: d = 14 + q; level n+1: d = q - 13) the mirror images.  Only they
// can be written by the chunk before a point's own.
template <bool kUpper>
__device__ __forceinline__ bool dep_nbr(int q) {
  return kUpper ? (q == 0 || q == 1 || q == 4 || q == 13) : (q == 26 || q == 35 || q == 38 || q == 39);
}

template <typename S, bool SMEM>
__global__ void __launch_bounds__(solve_threads_max<S>(), 2) ras_solve(
    const BoxDesc* __restrict__ boxes, const Chunk* __restrict__ chunks, const S* __restrict__ F,
    typename SolveArith<S>::type* __restrict__ V, const double* __restrict__ r, double* __restrict__ z,
    const int2* __restrict__ gtab, const int2* __restrict__ otab, const int* __restrict__ vtab, int bstride,
    int nstage, int* __restrict__ status, const int* gate, int gate_stride) {
  using T = typename SolveArith<S>::type;
  // the box's problem gate (one problem: gate_stride 0, every box reads gate[0])
  if (gate != nullptr && gate[boxes[blockIdx.x].prob * gate_stride] == 0) return;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + 1536);
  int* abort_at = reinterpret_cast<int*>(smem + 1536 + 8 * kMaxStages);   // block whose wait gave up, or -1
  S* buf0 = reinterpret_cast<S*>(smem + kSolveHeader);   // nstage buffers of bstride values
                                                        // (kLRanks x the largest chunk row stride)
  const BoxDesc bx = boxes[blockIdx.x];
  const long long P = bx.P;
  const S* Fb = F + bx.foff;
  const int px = bx.lx + 2, py = bx.ly + 2, pz = bx.lz + 2;
  const long long sy = px, sz = (long long)px * py, st = (long long)px * py * pz;
  const long long npad = kVecWidth * st * (bx.lt + 2);
  T* v = SMEM ? reinterpret_cast<T*>(buf0 + (size_t)nstage * bstride) : V + bx.voff;
  const int nch = bx.cend - bx.cbeg;
  const Chunk* ck = chunks + bx.cbeg;
  const int lane = threadIdx.x & (kLanes - 1), j = threadIdx.x / kLanes;
  // offsets of the lane's neighbours in the padded local vector
  int offL[kNbrPerLane], offU[kNbrPerLane];
#pragma unroll
  for (int i = 0; i < kNbrPerLane; ++i) {
    const int q = lane + kLanes * i;
    // earlier neighbour q: level n-1, spatial offset d = q (q < 27); level n, d = q - 27
    const int dl = q < 27 ? q : q - 27, tl = q < 27 ? -1 : 0;
    // later neighbour q: level n, d = 14 + q (q < 13); level n+1, d = q - 13
    const int du = q < 13 ? 14 + q : q - 13, tu = q < 13 ? 0 : 1;
    offL[i] = (int)(kVecWidth * ((dl % 3 - 1) + sy * ((dl / 3) % 3 - 1) + sz * (dl / 9 - 1) + st * tl));
    offU[i] = (int)(kVecWidth * ((du % 3 - 1) + sy * ((du / 3) % 3 - 1) + sz * (du / 9 - 1) + st * tu));
  }
  if (threadIdx.x == 0) {
    for (int b = 0; b < nstage; ++b) mbar_init(&bar[b], 1);
    mbar_fence_init();
    *abort_at = -1;
  }
  if (SMEM)
    for (long long i = threadIdx.x; i < npad; i += blockDim.x) v[i] = (T)0;
  __syncthreads();
  // The factor blocks stream in the order L(0), ..., L(nch-1), U(nch-1), ...,
  // U(0) through a ring of `nstage` buffers: block g goes to buffer g mod
  // nstage and is copied nstage - 1 steps before it is used.
  const int nblk = 2 * nch;
  auto chunk_of = [&](int g) { return g < nch ? g : nblk - 1 - g; };
  auto issue = [&](const Chunk& c, int g) {
    const bool upper = g >= nch;
    const int b = g % nstage;
    const unsigned rows = upper ? kURanks : kLRanks;
    const unsigned bytes = rows * (unsigned)c.cp * (unsigned)sizeof(S);
    const S* src = Fb + c.off + (upper ? (long long)kLRanks * c.cp : 0);
    fence_proxy_async();
    mbar_expect_tx(&bar[b], bytes);
    bulk_g2s(buf0 + (size_t)b * bstride, src, bytes, &bar[b]);
  };
  Chunk iss;   // thread 0: descriptor of the next block to copy
  if (threadIdx.x == 0) {
    for (int g = 0; g < min(nstage - 1, nblk); ++g) issue(ck[chunk_of(g)], g);
    if (nstage - 1 < nblk) iss = ck[chunk_of(nstage - 1)];
  }
  // gather R^delta r into the padded local vector while the first blocks arrive
  // (gtab: per box point, its global unknown index and its padded offset)
  for (int q = threadIdx.x; q < (int)P; q += blockDim.x) {
    const int2 e = gtab[bx.poff + q];
    st3(v + e.y, (T)r[e.x], (T)r[e.x + 1], (T)r[e.x + 2]);
  }
  __syncthreads();
  // Step g works on the chunk of block g (`cur`).  The descriptor of the
  // chunk after next and the point index of the next chunk are loaded one
  // step ahead, so the only loads left between a barrier and the arithmetic
  // are the vector's.  Steps 0..nch-1 are the forward sweep with the unit
  // lower factor, steps nch..2 nch-1 the backward sweep with the upper factor.
  Chunk cur, nxt;
  int vq_cur = 0;
  // neighbour values of the step; `pre`: the previous step already loaded the
  // ones that cannot change during it (see the end of the step)
  T nc[kNbrPerLane], ng[kNbrPerLane], nf[kNbrPerLane];
  bool pre = false;
  if (nblk > 0) {
    cur = ck[0];
    nxt = ck[chunk_of(min(1, nblk - 1))];
    vq_cur = j < cur.n ? vtab[bx.poff + cur.q0 + j] : 0;
  }
  // one step of either sweep; false when a copy wait gave up (the CTA stops)
  // kCp: the row stride of the chunk's block as a compile-time constant (a
  // full chunk: kCp = CH, so every factor read is [base + immediate]), or 0 for
  // the run-time stride of a ragged chunk
  auto step = [&](int g, auto upper_tag, auto cp_tag) -> bool {
    constexpr bool kUpper = decltype(upper_tag)::value;
    constexpr int kCp = decltype(cp_tag)::value;
    const int b = g % nstage;
    if (threadIdx.x == 0 && g + nstage - 1 < nblk) {
      issue(iss, g + nstage - 1);
      if (g + nstage < nblk) iss = ck[chunk_of(g + nstage)];
    }
    const Chunk nn = ck[chunk_of(min(g + 2, nblk - 1))];
    const int vq_nxt = (g + 1 < nblk && j < nxt.n) ? vtab[bx.poff + nxt.q0 + j] : 0;
    const Chunk& c = cur;
    const bool act = j < c.n;
    const int cp = kCp ? kCp : c.cp;
    T* vp = v + (act ? vq_cur : 0);
    // all neighbour loads of the step first (they depend on the previous steps
    // only, so they are in flight while the factor block is awaited), then the
    // arithmetic
    T v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
    for (int i = 0; i < kNbrPerLane; ++i) {
      if (!pre || dep_nbr<kUpper>(lane + kLanes * i)) {
        nc[i] = ng[i] = nf[i] = (T)0;
        if (act) ld3(vp + (kUpper ? offU[i] : offL[i]), nc[i], ng[i], nf[i]);
      }
    }
    if (act) ld3(vp, v0, v1, v2);
    if (!mbar_wait(&bar[b], (unsigned)(g / nstage) & 1u, status)) *abort_at = g;
    const S* B = buf0 + (size_t)b * bstride;
    T sc = 0, sg = 0, sf = 0;
    if constexpr (!kUpper) {
      if constexpr (sizeof(T) == 8) {
        // FP64: one FMA per product into two chains per sum (the FP64 pipe
        // is the limit: a product pair costs 2 operations instead of 3)
        T sc1 = 0, sf1 = 0;
#pragma unroll
        for (int i = 0; i < kNbrPerLane; ++i) {
          const int q = lane + kLanes * i;
          const S* rc = B + (2 * q) * cp + j;
          const S* rf = B + (94 + 2 * q) * cp + j;
          sc = fma(arith<T>(rc[0]), nc[i], sc);
          sc1 = fma(arith<T>(rc[cp]), nf[i], sc1);
          sf = fma(arith<T>(rf[0]), ng[i], sf);
          sf1 = fma(arith<T>(rf[cp]), nf[i], sf1);
          if (q >= 27) sg = fma(arith<T>(B[(80 + q - 27) * cp + j]), ng[i], sg);
        }
        sc += sc1;
        sf += sf1;
      } else {
#pragma unroll
        for (int i = 0; i < kNbrPerLane; ++i) {
          const int q = lane + kLanes * i;
          const S* rc = B + (2 * q) * cp + j;
          const S* rf = B + (94 + 2 * q) * cp + j;
          sc += arith<T>(rc[0]) * nc[i] + arith<T>(rc[cp]) * nf[i];
          sf += arith<T>(rf[0]) * ng[i] + arith<T>(rf[cp]) * nf[i];
          if (q >= 27) sg += arith<T>(B[(80 + q - 27) * cp + j]) * ng[i];
        }
      }
      sc = lane_sum(sc);
      sg = lane_sum(sg);
      sf = lane_sum(sf);
      // own-point terms in C, G, f order: the G row's own-C slot (row 93) and
      // the f row's own-G slot (row 174)
      if (act && lane == 0) {
        const T yc = v0 - sc;
        const T yg = v1 - sg - arith<T>(B[93 * cp + j]) * yc;
        const T yf = v2 - sf - arith<T>(B[174 * cp + j]) * yg;
        st3(vp, yc, yg, yf);
      }
    } else {
      T sf1 = 0;   // FP64: the f-row products in two FMA chains
#pragma unroll
      for (int i = 0; i < kNbrPerLane; ++i) {
        const int q = lane + kLanes * i;
        const S* rf = B + (71 + 2 * q) * cp + j;
        if constexpr (sizeof(T) == 8) {
          sf = fma(arith<T>(rf[0]), ng[i], sf);
          sf1 = fma(arith<T>(rf[cp]), nf[i], sf1);
        } else {
          sf += arith<T>(rf[0]) * ng[i] + arith<T>(rf[cp]) * nf[i];
        }
        if (q < 13) {
          const S* rc = B + (2 + 2 * q) * cp + j;
          if constexpr (sizeof(T) == 8)
            sc = fma(arith<T>(rc[cp]), nf[i], fma(arith<T>(rc[0]), nc[i], sc));
          else
            sc += arith<T>(rc[0]) * nc[i] + arith<T>(rc[cp]) * nf[i];
          sg += arith<T>(B[(29 + q) * cp + j]) * ng[i];
        } else {
          const int d = q - 13;
          sg += arith<T>(B[(42 + d + (d >= 13 ? 1 : 0)) * cp + j]) * ng[i];
          if (d == 13) sg += arith<T>(B[55 * cp + j]) * nc[i];
        }
      }
      sf += sf1;
      sc = lane_sum(sc);
      sg = lane_sum(sg);
      sf = lane_sum(sf);
      // the diagonal rows 0, 28, 70 hold the reciprocals of the pivots; the C
      // row's own-f slot (U row 1) is applied after the f row is solved
      if (act && lane == 0) {
        const T zf = (v2 - sf) * arith<T>(B[70 * cp + j]);
        const T zg = (v1 - sg) * arith<T>(B[28 * cp + j]);
        const T zc = (v0 - sc - arith<T>(B[1 * cp + j]) * zf) * arith<T>(B[0 * cp + j]);
        st3(vp, zc, zg, zf);
      }
    }
    // The next step's neighbours in the same sweep, except the few one
    // wavefront away (they may be points of this chunk), cannot change during
    // this step: with FP64 factors, load them now, so their latency overlaps
    // the barrier (measured at 32^3 x 64: the FP64 form 3 % faster; the FP32
    // solve 17 % slower, so FP32 and BF16 factors load after the barrier).
    pre = sizeof(S) == 8 && g + 1 < nblk && g + 1 != nch;
    if (pre) {
      const bool act2 = j < nxt.n;
      const T* vp2 = v + (act2 ? vq_nxt : 0);
#pragma unroll
      for (int i = 0; i < kNbrPerLane; ++i) {
        if (dep_nbr<kUpper>(lane + kLanes * i)) continue;
        nc[i] = ng[i] = nf[i] = (T)0;
        if (act2) ld3(vp2 + (kUpper ? offU[i] : offL[i]), nc[i], ng[i], nf[i]);
      }
    }
    __syncthreads();
    cur = nxt;
    nxt = nn;
    vq_cur = vq_nxt;
    return *abort_at < 0;
  };
  // forward sweep (unit lower factor), then backward sweep (upper factor)
  bool ok = true;
  using FullCp = std::integral_constant<int, ChunkCfg<S>::CH>;   // == chunk_stride(CH): no padding
  using AnyCp = std::integral_constant<int, 0>;
  const int full_cp = chunk_stride_dev<S>(ChunkCfg<S>::CH);
  for (int g = 0; ok && g < nch; ++g)
    ok = cur.cp == full_cp && full_cp == FullCp::value ? step(g, std::false_type{}, FullCp{})
                                                       : step(g, std::false_type{}, AnyCp{});
  for (int g = nch; ok && g < nblk; ++g)
    ok = cur.cp == full_cp && full_cp == FullCp::value ? step(g, std::true_type{}, FullCp{})
                                                       : step(g, std::true_type{}, AnyCp{});
  if (!ok) {
    // A wait gave up at block gf (status 2 is set): the blocks gf .. gf +
    // nstage - 1 may still be in flight into this CTA's buffers.  Thread 0
    // waits for them, again with the time limit, and the CTA returns without
    // writing z.
    if (threadIdx.x == 0) {
      const int gf = *abort_at;
      for (int q = gf; q < min(gf + nstage, nblk); ++q)
        mbar_wait(&bar[q % nstage], (unsigned)(q / nstage) & 1u, status);
    }
    return;
  }
  // scatter the owned part: (R^0)^T (otab: the owned points' global indices and offsets)
  for (int q = threadIdx.x; q < bx.nown; q += blockDim.x) {
    const int2 e = otab[bx.ooff + q];
    T a0, a1, a2;
    ld3(v + e.y, a0, a1, a2);
    z[e.x] = (double)a0;
    z[e.x + 1] = (double)a1;
    z[e.x + 2] = (double)a2;
  }
}

std::vector<std::pair<int, int>> parts(int n, int p) {
  std::vector<std::pair<int, int>> out;
  const int base = n / p, extra = n % p;
  int s = 0;
  for (int k = 0; k < p; ++k) {
    const int e = s + base + (k < extra ? 1 : 0);
    out.emplace_back(s, e);
    s = e;
  }
  return out;
}

// esz: bytes of a stored factor value, vsz: of a local-vector value
size_t solve_smem(int cpmax, int nstage, size_t esz, size_t vsz, long long max_pad, bool smem_vec) {
  const size_t bufs = (size_t)nstage * kLRanks * cpmax * esz;
  return kSolveHeader + bufs + (smem_vec ? (size_t)max_pad * vsz : 0);
}

// Chunk size, copy-ring depth and local-vector placement of the subdomain
// solve.  Each box is one CTA that steps through its chunks one after the
// other, so a step's latency decides the time.  The order of preference, as
// measured on GB300 (32^3 x 64 fine boxes, coarse-sized boxes, FP32 and
// FP64): the fewest waves of CTAs over the SMs (the runtime's occupancy for
// the shared memory, threads and registers); the local vectors in global
// memory (cached in L1) rather than in shared memory; the shallowest ring (a
// deeper ring takes shared memory from the L1 that caches the local
// vectors); the largest chunk (fewest steps).  ras_autotune measures instead.
struct SolveShape {
  int ch, cpmax, nstage, lanes;
  bool smem_vec;
};
template <typename T, bool SMEM>
const void* solve_kernel() {
  return (const void*)ras_solve<T, SMEM>;
}
// A requested shape (ras_setup_shape): 0 in a field leaves it to the chooser.
struct ShapeRequest {
  int ch = 0, nstage = 0, lanes = 0, place = 0;   // place: 1 shared-memory vector, 2 global-memory vector
};
// Picks the best shape allowed by `req`; KKT_ERR_ARG when none is.
template <typename T>
kkt_status choose_solve_shape(int nbox, long long max_pad, int nsm, const ShapeRequest& req, SolveShape* out) {
  if (req.lanes != 0 && req.lanes != kLanes) {
    set_error("ras_setup: the subdomain solve runs 4 lanes per point");
    return KKT_ERR_ARG;
  }
  const int cands[3] = {ChunkCfg<T>::CH, ChunkCfg<T>::CH2, ChunkCfg<T>::CH3};
  KKT_TRY_CUDA(cudaFuncSetAttribute(ras_solve<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemLimit));
  KKT_TRY_CUDA(cudaFuncSetAttribute(ras_solve<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemLimit));
  SolveShape best{};
  long long best_key = -1;
  for (int ci = 0; ci < 3; ++ci)
    for (int ns = 2; ns <= kMaxStages; ++ns)
      for (int sv = 1; sv >= 0; --sv) {
        const int ch = cands[ci], cp = chunk_stride<T>(ch);
        if ((req.ch && req.ch != ch) || (req.nstage && req.nstage != ns) || (req.place == 1 && !sv) ||
            (req.place == 2 && sv))
          continue;
        const size_t sm = solve_smem(cp, ns, sizeof(T), sizeof(typename SolveArith<T>::type), max_pad, sv != 0);
        if (sm > kSmemLimit) continue;
        const int threads = (ch * kLanes + 31) / 32 * 32;
        int per_sm = 0;
        KKT_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, sv ? solve_kernel<T, true>() : solve_kernel<T, false>(), threads, sm));
        if (per_sm < 1) continue;
        const long long waves = (nbox + (long long)nsm * per_sm - 1) / ((long long)nsm * per_sm);
        // smaller key is better: fewest waves, then the local vectors in global
        // memory (measured faster than in shared memory with this kernel, also on
        // the small coarse-level boxes: 0.285 vs 0.354 ms at 17^3 x 33 nodes, 4^4
        // boxes, overlap 1), the shallowest ring, the largest chunk
        const long long key = waves * 100000000LL + (sv ? 1000000 : 0) + (ns - 2) * 1000 + (100 - ch);
        if (best_key < 0 || key < best_key) {
          best_key = key;
          best = SolveShape{ch, cp, ns, kLanes, sv != 0};
        }
      }
  if (best_key < 0) {
    set_error("ras_setup: no subdomain-solve shape fits the request (chunk size, ring depth and vector "
              "placement must be a compiled combination that fits in shared memory)");
    return KKT_ERR_ARG;
  }
  *out = best;
  return KKT_OK;
}

}  // namespace

kkt_status ras_create(kkt_problem* const* probs, int nprob, const int nsub[4], int overlap, int local,
                      int factor_prec, const int* shape, ras_precond** out) {
  if (!probs || nprob < 1 || !nsub || !out) {
    set_error("ras_setup: null argument or no problem");
    return KKT_ERR_ARG;
  }
  *out = nullptr;
  for (int k = 0; k < nprob; ++k) {
    const kkt_problem* pk = probs[k];
    if (!pk) {
      set_error("ras_setup: null problem");
      return KKT_ERR_ARG;
    }
    const int dk[4] = {pk->nx, pk->ny, pk->nz, pk->L};
    for (int a = 0; a < 4; ++a)
      if (nsub[a] < 1 || nsub[a] > dk[a]) {
        set_error("ras_setup: each nsub must lie in [1, points along that axis]");
        return KKT_ERR_ARG;
      }
  }
  if (nprob > 1 && local != 0) {
    set_error("ras_setup_batch: the subdomains of several problems use ILU(0) local solves");
    return KKT_ERR_ARG;
  }
  kkt_problem* p = probs[0];
  if (overlap < 0 || local < 0 || local > 3 || (factor_prec != 64 && factor_prec != 32 && factor_prec != 16)) {
    set_error("ras_setup: overlap must be >= 0, local 0 (ILU(0)), 1 (exact LU), 2 (ILU(1)) or 3 (point-block "
              "ILU(0)), factor_prec 64, 32 or 16");
    return KKT_ERR_ARG;
  }
  if (local == 1 && factor_prec != 64) {
    set_error("ras_setup: the exact local LU is FP64 only (factor_prec 64)");
    return KKT_ERR_ARG;
  }
  if (local >= 2 && factor_prec == 16) {
    set_error("ras_setup: ILU(1) and point-block ILU(0) factor in FP64 or FP32 (factor_prec 64 or 32)");
    return KKT_ERR_ARG;
  }
  const SlotTables& T = tables();
  {
    long long h = 0;
    for (int i = 0; i < kSlots; ++i)
      h = (h * 131 + (i + 1) * (T.dt[i] + 2) * 7 + (T.dz[i] + 2) * 11 + (T.dy[i] + 2) * 13 + (T.dx[i] + 2) * 17 +
           T.comp[i] * 19) % 1000000007LL;
    if (h != kGenSlotChecksum || kGenRowSlots0 != T.count[0] || kGenRowSlots1 != T.count[1] ||
        kGenRowSlots2 != T.count[2]) {
      set_error("ras_setup: generated elimination code does not match the slot tables");
      return KKT_ERR_ARG;
    }
    for (int i = 0; i < kSlots; ++i)
      if (kGenRank[i] != slot_rank(i)) {
        set_error("ras_setup: generated elimination code does not match the chunk block order");
        return KKT_ERR_ARG;
      }
  }
  if (T.base[0] != kCBase || T.diag[0] != kCDiag || T.base[1] != kGBase || T.diag[1] != kGDiag ||
      T.base[2] != kFBase || T.diag[2] != kFDiag || T.base[2] + T.count[2] != kFEnd) {
    set_error("ras_setup: internal slot table mismatch");
    return KKT_ERR_ARG;
  }

  ras_precond* m = new (std::nothrow) ras_precond();
  if (!m) return KKT_ERR_NOMEM;
  m->prob = p;
  m->probs.assign(probs, probs + nprob);
  m->vec_off.assign(1, 0);
  for (int k = 0; k < nprob; ++k) m->vec_off.push_back(m->vec_off.back() + probs[k]->n);
  m->n_total = m->vec_off.back();
  m->prec = factor_prec;
  m->local = local;
  auto stride = [&](int n) { return chunk_stride_of(factor_prec, n); };
  // every box: its problem and the owned part of each axis (part k of n holds
  // floor(n/p) + (k < n mod p)); the extended box adds `overlap`, trimmed
  struct Geom {
    int prob;
    std::pair<int, int> own[4];
    long long points;
  };
  std::vector<Geom> geoms;
  for (int k = 0; k < nprob; ++k) {
    const kkt_problem* pk = probs[k];
    const int dk[4] = {pk->nx, pk->ny, pk->nz, pk->L};
    std::vector<std::pair<int, int>> prk[4];
    for (int a = 0; a < 4; ++a) prk[a] = parts(dk[a], nsub[a]);
    for (int it = 0; it < nsub[3]; ++it)
      for (int iz = 0; iz < nsub[2]; ++iz)
        for (int iy = 0; iy < nsub[1]; ++iy)
          for (int ix = 0; ix < nsub[0]; ++ix) {
            Geom g{k, {prk[0][ix], prk[1][iy], prk[2][iz], prk[3][it]}, 1};
            for (int a = 0; a < 4; ++a)
              g.points *= std::min(dk[a], g.own[a].second + overlap) - std::max(0, g.own[a].first - overlap);
            geoms.push_back(g);
          }
  }
  // several problems: the largest boxes first, so that the CTAs of one launch
  // (one per box, started in list order) finish as close together as they can
  if (nprob > 1)
    std::stable_sort(geoms.begin(), geoms.end(), [](const Geom& a, const Geom& b) { return a.points > b.points; });
  {
    // largest padded local vector
    long long pad = 0;
    for (const Geom& g : geoms) {
      const kkt_problem* pk = probs[g.prob];
      const int dk[4] = {pk->nx, pk->ny, pk->nz, pk->L};
      long long v = kVecWidth;
      for (int a = 0; a < 4; ++a)
        v *= std::min(dk[a], g.own[a].second + overlap) - std::max(0, g.own[a].first - overlap) + 2;
      pad = std::max(pad, v);
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
      cudaGetLastError();
      set_error("ras_setup: cannot query the current device");
      delete m;
      return KKT_ERR_CUDA;
    }
    const int nbox = (int)geoms.size();
    ShapeRequest req;
    if (shape) {
      req.ch = shape[0];
      req.nstage = shape[1];
      req.lanes = shape[2];
      req.place = shape[3];
    }
    SolveShape sh{};
    const kkt_status cs = factor_prec == 64   ? choose_solve_shape<double>(nbox, pad, nsm, req, &sh)
                          : factor_prec == 32 ? choose_solve_shape<float>(nbox, pad, nsm, req, &sh)
                                              : choose_solve_shape<__nv_bfloat16>(nbox, pad, nsm, req, &sh);
    if (cs != KKT_OK) {
      delete m;
      return cs;
    }
    m->ch = sh.ch;
    m->cpmax = sh.cpmax;
    m->smem_vec = sh.smem_vec;
    m->nstage = sh.nstage;
    m->lanes = sh.lanes;
  }
  const int CH = m->ch;
  std::vector<BoxDesc> boxes;
  std::vector<int> perm, iperm, lptr;
  std::vector<int2> ptab, gtab, otab;
  std::vector<int> vtab;
  if (m->n_total >= INT32_MAX) {
    set_error("ras_setup: more than 2^31 unknowns are not supported");
    delete m;
    return KKT_ERR_ARG;
  }
  std::vector<Chunk> chunks;
  long long foff = 0, voff = 0;
  for (const Geom& geo : geoms) {
          const kkt_problem* pk = probs[geo.prob];
          const long long gbase = m->vec_off[geo.prob];   // the problem's first unknown
          const int dims[4] = {pk->nx, pk->ny, pk->nz, pk->L};
          BoxDesc b{};
          b.prob = geo.prob;
          const std::pair<int, int>* own[4] = {&geo.own[0], &geo.own[1], &geo.own[2], &geo.own[3]};
          int lo[4], hi[4];
          for (int a = 0; a < 4; ++a) {
            lo[a] = std::max(0, own[a]->first - overlap);
            hi[a] = std::min(dims[a], own[a]->second + overlap);
          }
          b.x0 = lo[0]; b.y0 = lo[1]; b.z0 = lo[2]; b.t0 = lo[3];
          b.lx = hi[0] - lo[0]; b.ly = hi[1] - lo[1]; b.lz = hi[2] - lo[2]; b.lt = hi[3] - lo[3];
          b.ox0 = own[0]->first; b.ox1 = own[0]->second; b.oy0 = own[1]->first; b.oy1 = own[1]->second;
          b.oz0 = own[2]->first; b.oz1 = own[2]->second; b.ot0 = own[3]->first; b.ot1 = own[3]->second;
          b.P = (long long)b.lx * b.ly * b.lz * b.lt;
          b.nlev = (b.lx - 1) + 2 * (b.ly - 1) + 4 * (b.lz - 1) + 8 * (b.lt - 1) + 1;
          b.foff = foff;
          b.voff = voff;
          b.poff = (long long)perm.size();
          b.loff = (long long)lptr.size();
          voff += (long long)kVecWidth * (b.lx + 2) * (b.ly + 2) * (b.lz + 2) * (b.lt + 2);
          // counting sort of the points by wavefront
          std::vector<int> cnt(b.nlev + 1, 0);
          for (int kt = 0; kt < b.lt; ++kt)
            for (int kz = 0; kz < b.lz; ++kz)
              for (int ky = 0; ky < b.ly; ++ky)
                for (int kx = 0; kx < b.lx; ++kx) cnt[kx + 2 * ky + 4 * kz + 8 * kt + 1]++;
          for (int w = 0; w < b.nlev; ++w) cnt[w + 1] += cnt[w];
          for (int w = 0; w <= b.nlev; ++w) lptr.push_back(cnt[w]);
          std::vector<int> bp(b.P), bi(b.P);
          std::vector<int> fill(cnt.begin(), cnt.end() - 1);
          int lex = 0;
          for (int kt = 0; kt < b.lt; ++kt)
            for (int kz = 0; kz < b.lz; ++kz)
              for (int ky = 0; ky < b.ly; ++ky)
                for (int kx = 0; kx < b.lx; ++kx, ++lex) {
                  const int q = fill[kx + 2 * ky + 4 * kz + 8 * kt]++;
                  bp[q] = lex;
                  bi[lex] = q;
                }
          perm.insert(perm.end(), bp.begin(), bp.end());
          iperm.insert(iperm.end(), bi.begin(), bi.end());
          // index tables of the solve: global index and padded offset of every
          // point (lexicographic), padded offset in wavefront order, owned points
          {
            const long long sy = b.lx + 2, sz = sy * (b.ly + 2), st = sz * (b.lz + 2);
            auto pad = [&](int kx, int ky, int kz, int kt) {
              return (int)(kVecWidth * ((kx + 1) + sy * (ky + 1) + sz * (kz + 1) + st * (kt + 1)));
            };
            auto glob = [&](int kx, int ky, int kz, int kt) {
              return (int)(gbase + 3 * ((long long)(b.t0 + kt) * pk->N + (b.x0 + kx) +
                                        (long long)pk->nx * ((b.y0 + ky) + (long long)pk->ny * (b.z0 + kz))));
            };
            const size_t g0 = gtab.size();
            gtab.resize(g0 + b.P);
            vtab.resize(g0 + b.P);
            int q = 0;
            for (int kt = 0; kt < b.lt; ++kt)
              for (int kz = 0; kz < b.lz; ++kz)
                for (int ky = 0; ky < b.ly; ++ky)
                  for (int kx = 0; kx < b.lx; ++kx, ++q) gtab[g0 + q] = make_int2(glob(kx, ky, kz, kt), pad(kx, ky, kz, kt));
            for (int w = 0; w < (int)b.P; ++w) vtab[g0 + w] = gtab[g0 + bp[w]].y;
            b.ooff = (long long)otab.size();
            for (int gt = b.ot0; gt < b.ot1; ++gt)
              for (int gz = b.oz0; gz < b.oz1; ++gz)
                for (int gy = b.oy0; gy < b.oy1; ++gy)
                  for (int gx = b.ox0; gx < b.ox1; ++gx)
                    otab.push_back(make_int2(glob(gx - b.x0, gy - b.y0, gz - b.z0, gt - b.t0),
                                             pad(gx - b.x0, gy - b.y0, gz - b.z0, gt - b.t0)));
            b.nown = (int)((long long)otab.size() - b.ooff);
          }
          // chunks of each wavefront and the storage offset of every point
          b.cbeg = (int)chunks.size();
          const size_t pt0 = ptab.size();
          ptab.resize(pt0 + b.P);
          long long off = 0;
          for (int w = 0; w < b.nlev; ++w)
            for (int q0 = cnt[w]; q0 < cnt[w + 1]; q0 += CH) {
              Chunk c{};
              c.box = (int)boxes.size();
              c.w = w;
              c.q0 = q0;
              c.n = std::min(CH, cnt[w + 1] - q0);
              c.cp = stride(c.n);
              c.off = off;
              for (int k = 0; k < c.n; ++k) ptab[pt0 + q0 + k] = make_int2((int)(off + k), c.cp);
              off += (long long)kSlots * c.cp;
              chunks.push_back(c);
            }
          b.cend = (int)chunks.size();
          // the unit row of pivot points outside the box, padded so that the
          // next box's blocks start on a 16-byte boundary (bulk copies need it)
          b.unit = off;
          off += kUnitRowSpan;
          if (off > INT32_MAX) {
            set_error("ras_setup: a subdomain holds more than 2^31 factor values; use more subdomains");
            delete m;
            return KKT_ERR_ARG;
          }
          foff += off;
          if (local == 1) {
            // exact LU: band of the box matrix in natural point-block order
            const long long n_b = 3 * b.P;
            b.kl = 3 * (1 + b.lx + b.lx * b.ly + b.lx * b.ly * b.lz) + 2;
            if (b.kl > kMaxLuBand || n_b > kMaxLuUnknowns) {
              set_error("ras_setup: a subdomain is too large for the exact local LU (at most " +
                        std::to_string(kMaxLuUnknowns) + " unknowns and half-bandwidth " +
                        std::to_string(kMaxLuBand) + "); use ILU(0) or more subdomains");
              delete m;
              return KKT_ERR_ARG;
            }
            b.aoff = m->ab_count;
            m->ab_count += n_b * (3LL * b.kl + 1);
          }
          boxes.push_back(b);
        }
  m->nbox = (int)boxes.size();
  m->nchunk = (int)chunks.size();
  m->boxes_h = boxes;
  m->fcount = foff;
  m->vcount = voff;
  m->max_pad = 0;
  for (const BoxDesc& b : boxes)
    m->max_pad = std::max(m->max_pad, (long long)kVecWidth * (b.lx + 2) * (b.ly + 2) * (b.lz + 2) * (b.lt + 2));
  // bytes of a stored factor value and of a local-vector value
  const size_t esz = factor_prec == 64 ? sizeof(double) : (factor_prec == 32 ? sizeof(float) : 2);
  const size_t vsz = factor_prec == 64 ? sizeof(double) : sizeof(float);
  // every bulk copy of the solve must start on a 16-byte boundary and move a
  // multiple of 16 bytes: check each chunk's L and U blocks before any launch
  for (const Chunk& c : chunks) {
    const long long base = (boxes[c.box].foff + c.off) * (long long)esz;
    const long long lbytes = (long long)kLRanks * c.cp * (long long)esz;
    const long long ubytes = (long long)kURanks * c.cp * (long long)esz;
    if (base % 16 || lbytes % 16 || ubytes % 16) {
      set_error("ras_setup: internal error: a factor block is not 16-byte aligned");
      delete m;
      return KKT_ERR_ARG;
    }
  }
  auto fail = [&](kkt_status st, const char* what) {
    cudaGetLastError();
    set_error(std::string("ras_setup: ") + what);
    ras_destroy(m);
    return st;
  };
  if (cudaMalloc(&m->boxes, boxes.size() * sizeof(BoxDesc)) != cudaSuccess ||
      cudaMalloc(&m->perm, perm.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->iperm, iperm.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->lptr, lptr.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->ptab, ptab.size() * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&m->gtab, gtab.size() * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&m->otab, std::max<size_t>(1, otab.size()) * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&m->vtab, vtab.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->chunks, chunks.size() * sizeof(Chunk)) != cudaSuccess ||
      cudaMalloc(&m->F, (local >= 2 ? 16 : foff) * esz) != cudaSuccess ||
      cudaMalloc(&m->V, (local >= 2 ? 16 : voff) * vsz) != cudaSuccess ||
      (factor_prec == 16 && cudaMalloc(&m->Ffac, foff * sizeof(float)) != cudaSuccess) ||
      cudaMalloc(&m->status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&m->dprobs, m->probs.size() * sizeof(DevProblem)) != cudaSuccess)
    return fail(KKT_ERR_NOMEM, "device allocation failed");
  m->dprobs_h.resize(m->probs.size());
  if (local == 1) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(KKT_ERR_CUDA, "cudaMemGetInfo failed");
    const double need = (double)m->ab_count * sizeof(double);
    if (need > 0.8 * (double)free_b)
      return fail(KKT_ERR_NOMEM, ("the exact local LU needs " + std::to_string((long long)(need / 1e6)) +
                                  " MB of band storage; use ILU(0) or more subdomains").c_str());
    if (cudaMalloc(&m->AB, m->ab_count * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->ipiv, 3 * perm.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&m->lu_ju, 2 * boxes.size() * sizeof(int)) != cudaSuccess)
      return fail(KKT_ERR_NOMEM, "device allocation failed (exact LU)");
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    m->lu_ctas = std::max(1, std::min(64, nsm / std::max(1, m->nbox)));   // one wave of 1024-thread CTAs
  }
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpy(m->boxes, boxes.data(), boxes.size() * sizeof(BoxDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->iperm, iperm.data(), iperm.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->lptr, lptr.data(), lptr.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->ptab, ptab.data(), ptab.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->gtab, gtab.data(), gtab.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !otab.empty())
    e = cudaMemcpy(m->otab, otab.data(), otab.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->vtab, vtab.data(), vtab.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->chunks, chunks.data(), chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->F, 0, (local >= 2 ? 16 : foff) * esz);
  if (e == cudaSuccess) e = cudaMemset(m->V, 0, (local >= 2 ? 16 : voff) * vsz);
  if (e == cudaSuccess && m->Ffac) e = cudaMemset(m->Ffac, 0, foff * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->status, 0, sizeof(int));
  if (e != cudaSuccess) return fail(KKT_ERR_CUDA, cudaGetErrorString(e));
  kkt_status st = local >= 2 ? gp_create(m, local, factor_prec) : KKT_OK;
  if (st == KKT_OK) st = ras_factor(m, nullptr);
  if (st != KKT_OK) {
    ras_destroy(m);
    return st;
  }
  *out = m;
  return KKT_OK;
}

namespace {

template <typename S>
kkt_status launch_solve(ras_precond* m, const double* r, double* z, typename SolveArith<S>::type* V,
                        cudaStream_t s, const int* gate = nullptr, int gate_stride = 0) {
  using T = typename SolveArith<S>::type;
  const int threads = (m->ch * kLanes + 31) / 32 * 32;
  const int bstride = kLRanks * m->cpmax;
  // (the dynamic shared-memory limit of both instances is raised at set-up, in choose_solve_shape)
  const size_t smem = solve_smem(m->cpmax, m->nstage, sizeof(S), sizeof(T), m->max_pad, m->smem_vec);
  if (m->smem_vec)
    ras_solve<S, true><<<m->nbox, threads, smem, s>>>(m->boxes, m->chunks, (const S*)m->F, V, r, z, m->gtab,
                                                      m->otab, m->vtab, bstride, m->nstage, m->status, gate,
                                                      gate_stride);
  else
    ras_solve<S, false><<<m->nbox, threads, smem, s>>>(m->boxes, m->chunks, (const S*)m->F, V, r, z, m->gtab,
                                                       m->otab, m->vtab, bstride, m->nstage, m->status, gate,
                                                       gate_stride);
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

}  // namespace

kkt_status ras_factor_enqueue(ras_precond* m, cudaStream_t s) {
  KKT_TRY_CUDA(cudaMemsetAsync(m->status, 0, sizeof(int), s));
  // the problems as the value gather reads them now (the regularisation may have changed)
  for (size_t k = 0; k < m->probs.size(); ++k) m->dprobs_h[k] = m->probs[k]->dev();
  KKT_TRY_CUDA(cudaMemcpyAsync(m->dprobs, m->dprobs_h.data(), m->dprobs_h.size() * sizeof(DevProblem),
                               cudaMemcpyHostToDevice, s));
  if (m->gp) KKT_TRY(gp_factor(m, s));
  else if (m->local == 1) KKT_TRY(ras_lu_factor(m, s));
  else if (m->prec == 64) KKT_TRY(ras_factor_launch64(m, s));
  else if (m->prec == 32) KKT_TRY(ras_factor_launch32(m, s));
  else KKT_TRY(ras_factor_launch16(m, s));
  return KKT_OK;
}

kkt_status ras_factor_status(ras_precond* m) {
  int st = 0;
  KKT_TRY_CUDA(cudaMemcpy(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    set_error("ras_setup: zero or non-finite pivot in a subdomain factorisation");
    return KKT_ERR_ZERO_PIVOT;
  }
  return KKT_OK;
}

kkt_status ras_factor(ras_precond* m, cudaStream_t s) {
  KKT_TRY(ras_factor_enqueue(m, s));
  KKT_TRY_CUDA(cudaStreamSynchronize(s));
  return ras_factor_status(m);
}

kkt_status ras_launch(ras_precond* m, const double* r, double* z, cudaStream_t s, const int* gate,
                      int gate_stride) {
  TimedScope timed(&m->timing, s);
  if (m->gp) return gp_solve(m, r, z, s, gate);
  if (m->local == 1) return ras_lu_solve(m, r, z, s, gate);
  if (m->prec == 64) return launch_solve<double>(m, r, z, (double*)m->V, s, gate, gate_stride);
  if (m->prec == 32) return launch_solve<float>(m, r, z, (float*)m->V, s, gate, gate_stride);
  return launch_solve<__nv_bfloat16>(m, r, z, (float*)m->V, s, gate, gate_stride);
}

kkt_status ras_check(ras_precond* m) {
  int st = 0;
  KKT_TRY_CUDA(cudaMemcpy(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st == 2) {
    set_error("ras_apply: a subdomain solve gave up waiting for its factor copy");
    return KKT_ERR_CUDA;
  }
  return KKT_OK;
}

extern "C" kkt_status ras_setup(kkt_problem* p, const int nsub[4], int overlap, int local, int factor_prec,
                                ras_precond** out) {
  NvtxRange nvtx_("ras_setup");
  return ras_create(&p, 1, nsub, overlap, local, factor_prec, nullptr, out);
}

extern "C" kkt_status ras_setup_shape(kkt_problem* p, const int nsub[4], int overlap, int local, int factor_prec,
                                      const int shape[4], ras_precond** out) {
  if (!shape) {
    set_error("ras_setup_shape: null shape");
    return KKT_ERR_ARG;
  }
  if (shape[0] < 0 || shape[1] < 0 || (shape[1] != 0 && (shape[1] < 2 || shape[1] > kMaxStages)) ||
      (shape[2] != 0 && shape[2] != kLanes) || shape[3] < 0 || shape[3] > 2) {
    set_error("ras_setup_shape: shape = {chunk points >= 0, ring buffers 0 or 2..4, lanes 0 or 4, "
              "vector placement 0, 1 or 2}");
    return KKT_ERR_ARG;
  }
  return ras_create(&p, 1, nsub, overlap, local, factor_prec, shape, out);
}

extern "C" kkt_status ras_setup_batch(kkt_problem* const* probs, int nprob, const int nsub[4], int overlap,
                                      int factor_prec, const int shape[4], ras_precond** out) {
  if (shape && (shape[0] < 0 || shape[1] < 0 || (shape[1] != 0 && (shape[1] < 2 || shape[1] > kMaxStages)) ||
                (shape[2] != 0 && shape[2] != kLanes) || shape[3] < 0 || shape[3] > 2)) {
    set_error("ras_setup_batch: shape = {chunk points >= 0, ring buffers 0 or 2..4, lanes 0 or 4, "
              "vector placement 0, 1 or 2}");
    return KKT_ERR_ARG;
  }
  return ras_create(probs, nprob, nsub, overlap, 0, factor_prec, shape, out);
}

extern "C" kkt_status ras_apply(ras_precond* m, const double* r, double* z, void* stream) {
  NvtxRange nvtx_("ras_apply");
  if (!m || !r || !z) {
    set_error("ras_apply: null argument");
    return KKT_ERR_ARG;
  }
  if (spans_overlap(r, z, m->n_total)) {
    set_error("ras_apply: r and z must not overlap");
    return KKT_ERR_ARG;
  }
  return ras_launch(m, r, z, (cudaStream_t)stream);
}

extern "C" kkt_status ras_solve_shape(const ras_precond* m, int* chunk_points, int* stages, int* lanes,
                                      int* smem_vectors) {
  if (!m) {
    set_error("ras_solve_shape: null argument");
    return KKT_ERR_ARG;
  }
  if (chunk_points) *chunk_points = m->ch;
  if (stages) *stages = m->nstage;
  if (lanes) *lanes = m->lanes;
  if (smem_vectors) *smem_vectors = m->smem_vec ? 1 : 0;
  return KKT_OK;
}

extern "C" kkt_status ras_status(ras_precond* m, int* code, void* stream) {
  if (!m || !code) {
    set_error("ras_status: null argument");
    return KKT_ERR_ARG;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  int st = 0;
  KKT_TRY_CUDA(cudaMemcpyAsync(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  KKT_TRY_CUDA(cudaStreamSynchronize(s));
  *code = st;
  if (*code == 2) {
    set_error("ras_status: a subdomain solve gave up waiting for its factor copy");
    return KKT_ERR_CUDA;
  }
  if (*code == 1) {
    set_error("ras_status: zero or non-finite pivot in a subdomain factorisation");
    return KKT_ERR_ZERO_PIVOT;
  }
  return KKT_OK;
}

extern "C" kkt_status ras_selftest_wait(ras_precond* m, double limit_ms, void* stream) {
  if (!m || !(limit_ms > 0.0) || limit_ms > 1000.0) {
    set_error("ras_selftest_wait: null handle or limit_ms outside (0, 1000]");
    return KKT_ERR_ARG;
  }
  wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(m->status, (unsigned long long)(limit_ms * 1e6));
  KKT_COUNT(1);
  KKT_TRY_CUDA(cudaGetLastError());
  return KKT_OK;
}

extern "C" kkt_status ras_info(const ras_precond* m, int* nbox, long long* points, long long* factor_values,
                               int* value_bytes) {
  if (!m) {
    set_error("ras_info: null argument");
    return KKT_ERR_ARG;
  }
  long long pts = 0;
  for (const BoxDesc& b : m->boxes_h) pts += b.P;
  if (nbox) *nbox = m->nbox;
  if (points) *points = pts;
  if (factor_values) *factor_values = m->local == 1 ? m->ab_count : (m->gp ? gp_factor_count(m) : m->fcount);
  if (value_bytes) *value_bytes = m->prec == 64 ? 8 : (m->prec == 32 ? 4 : 2);
  return KKT_OK;
}

extern "C" kkt_status ras_refactor(ras_precond* m, void* stream) {
  NvtxRange nvtx_("ras_refactor");
  if (!m) {
    set_error("ras_refactor: null argument");
    return KKT_ERR_ARG;
  }
  return ras_factor(m, (cudaStream_t)stream);
}

extern "C" kkt_status ras_timing_read(ras_precond* m, int kernel, double* total_ms, long long* launches) {
  if (!m || (kernel != 0 && kernel != 1)) {
    set_error("ras_timing_read: null handle or kernel not 0 (solve) / 1 (factorisation)");
    return KKT_ERR_ARG;
  }
  TimingLog& log = kernel == 0 ? m->timing : m->factor_timing;
  log.drain();
  if (total_ms) *total_ms = log.total_ms;
  if (launches) *launches = log.count;
  return KKT_OK;
}

extern "C" kkt_status kkt_timing_reset(kkt_problem* p, ras_precond* m) {
  if (p) p->mv_timing.reset();
  if (m) {
    m->timing.reset();
    m->factor_timing.reset();
  }
  return KKT_OK;
}

extern "C" void ras_destroy(ras_precond* m) {
  if (!m) return;
  cudaFree(m->boxes);
  cudaFree(m->perm);
  cudaFree(m->iperm);
  cudaFree(m->lptr);
  cudaFree(m->ptab);
  cudaFree(m->gtab);
  cudaFree(m->otab);
  cudaFree(m->vtab);
  cudaFree(m->Ffac);
  cudaFree(m->AB);
  cudaFree(m->ipiv);
  cudaFree(m->lu_ju);
  cudaFree(m->chunks);
  cudaFree(m->F);
  cudaFree(m->V);
  cudaFree(m->status);
  cudaFree(m->dprobs);
  gp_destroy(m);
  delete m->bw;
  delete m;
}

// ---------------------------------------------------------------------------
// Allocation-free subdomain solve.  The padded local vectors the solve works
// in come from a fixed array compiled into the library instead of the handle.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;   // 32 MiB per device
__device__ __align__(256) unsigned char g_ras_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_ptr[64] = {};

// Device address of the static scratch on the current device, looked up once
// per device (the host-side symbol is only a stand-in for it).
kkt_status static_scratch(void** out) {
  int dev = 0;
  KKT_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("ras_apply_static: device ordinal out of range");
    return KKT_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_ras_static_scratch);
    if (e != cudaSuccess || !ptr) {
      set_error(std::string("ras_apply_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return KKT_ERR_CUDA;
    }
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return KKT_OK;
}

}  // namespace

extern "C" kkt_status ras_apply_static(ras_precond* m, const double* r, double* z, void* stream) {
  if (!m || !r || !z) {
    set_error("ras_apply_static: null argument");
    return KKT_ERR_ARG;
  }
  if (spans_overlap(r, z, m->n_total)) {
    set_error("ras_apply_static: r and z must not overlap");
    return KKT_ERR_ARG;
  }
  if (m->local != 0) {
    set_error("ras_apply_static: only ILU(0) preconditioners have a static-scratch apply; use ras_apply");
    return KKT_ERR_ARG;
  }
  void* scratch = nullptr;
  KKT_TRY(static_scratch(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  // A solve that keeps the local vectors in shared memory never reads the
  // scratch: no size limit and nothing to clear.
  if (!m->smem_vec) {
    const size_t bytes = (size_t)m->vcount * (m->prec == 64 ? sizeof(double) : sizeof(float));
    if (bytes > kStaticScratchBytes) {
      set_error("ras_apply_static: the subdomain local vectors need " + std::to_string(bytes) +
                " bytes, more than the " + std::to_string(kStaticScratchBytes) +
                "-byte static scratch; use ras_apply");
      return KKT_ERR_ARG;
    }
    // the ghost layers of the local vectors must read zero; earlier calls (on
    // any handle) may have left other data at those positions
    KKT_TRY_CUDA(cudaMemsetAsync(scratch, 0, bytes, s));
  }
  if (m->prec == 64) return launch_solve<double>(m, r, z, (double*)scratch, s);
  if (m->prec == 32) return launch_solve<float>(m, r, z, (float*)scratch, s);
  return launch_solve<__nv_bfloat16>(m, r, z, (float*)scratch, s);
}

// ---------------------------------------------------------------------------
// Autotuner of the subdomain solve's shape: every compiled chunk size with
// 2 and 3 copy buffers (local vectors placed as the chooser places them) is
// set up on the given problems and timed over `reps` applies with CUDA
// events; the fastest is returned and, with a cache file, remembered there
// under a key of the problems' sizes, the split, the precision and the
// device, one line per key ("key<TAB>chunk stages ms").
// ---------------------------------------------------------------------------
namespace {

std::string tune_key(kkt_problem* const* probs, int nprob, const int nsub[4], int overlap, int prec) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::string k = std::string(prop.name) + ";prec=" + std::to_string(prec) + ";ov=" + std::to_string(overlap) +
                  ";nsub=" + std::to_string(nsub[0]) + "," + std::to_string(nsub[1]) + "," + std::to_string(nsub[2]) +
                  "," + std::to_string(nsub[3]) + ";";
  for (int i = 0; i < nprob; ++i)
    k += std::to_string(probs[i]->nx) + "x" + std::to_string(probs[i]->ny) + "x" + std::to_string(probs[i]->nz) +
         "x" + std::to_string(probs[i]->L) + (i + 1 < nprob ? "," : "");
  for (char& c : k)
    if (c == '\t' || c == '\n') c = ' ';
  return k;
}

__global__ void fill_ones(double* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = 1.0;
}

}  // namespace

extern "C" kkt_status ras_autotune(kkt_problem* const* probs, int nprob, const int nsub[4], int overlap,
                                   int factor_prec, int reps, const char* cache_path, int shape_out[4],
                                   double* best_ms) {
  if (!probs || nprob < 1 || !nsub || !shape_out || reps < 1 ||
      (factor_prec != 64 && factor_prec != 32 && factor_prec != 16)) {
    set_error("ras_autotune: bad argument");
    return KKT_ERR_ARG;
  }
  const std::string key = tune_key(probs, nprob, nsub, overlap, factor_prec);
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[4096];
      while (std::fgets(line, sizeof(line), f)) {
        char* tab = std::strchr(line, '\t');
        if (!tab || std::string(line, tab) != key) continue;
        int ch = 0, ns = 0;
        double ms = 0.0;
        if (std::sscanf(tab + 1, "%d %d %lf", &ch, &ns, &ms) == 3) {
          std::fclose(f);
          shape_out[0] = ch;
          shape_out[1] = ns;
          shape_out[2] = kLanes;
          shape_out[3] = 0;
          if (best_ms) *best_ms = ms;
          return KKT_OK;
        }
      }
      std::fclose(f);
    }
  }
  int cands[3] = {ChunkCfg<float>::CH, ChunkCfg<float>::CH2, ChunkCfg<float>::CH3};
  if (factor_prec == 64) {
    cands[0] = ChunkCfg<double>::CH;
    cands[1] = ChunkCfg<double>::CH2;
    cands[2] = ChunkCfg<double>::CH3;
  } else if (factor_prec == 16) {
    cands[0] = ChunkCfg<__nv_bfloat16>::CH;
    cands[1] = ChunkCfg<__nv_bfloat16>::CH2;
    cands[2] = ChunkCfg<__nv_bfloat16>::CH3;
  }
  long long n = 0;
  for (int i = 0; i < nprob; ++i) n += probs[i]->n;
  double *r = nullptr, *z = nullptr;
  if (cudaMalloc(&r, n * sizeof(double)) != cudaSuccess || cudaMalloc(&z, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(r);
    set_error("ras_autotune: device allocation failed");
    return KKT_ERR_NOMEM;
  }
  fill_ones<<<1216, 256>>>(r, n);
  KKT_COUNT(1);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = -1.0;
  int best_ch = 0, best_ns = 0;
  kkt_status err = KKT_OK;
  for (int ci = 0; ci < 3 && err == KKT_OK; ++ci)
    for (int ns = 2; ns <= 3 && err == KKT_OK; ++ns) {
      const int shape[4] = {cands[ci], ns, 0, 0};
      ras_precond* m = nullptr;
      const kkt_status st = ras_create(probs, nprob, nsub, overlap, 0, factor_prec, shape, &m);
      if (st == KKT_ERR_ARG) continue;   // this shape does not fit the device
      if (st != KKT_OK) {
        err = st;
        break;
      }
      kkt_status ls = ras_launch(m, r, z, nullptr);   // warm-up
      cudaEventRecord(e0, nullptr);
      for (int i = 0; i < reps && ls == KKT_OK; ++i) ls = ras_launch(m, r, z, nullptr);
      cudaEventRecord(e1, nullptr);
      float ms = 0.f;
      if (ls == KKT_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        const double per = ms / reps;
        if (best < 0 || per < best) {
          best = per;
          best_ch = cands[ci];
          best_ns = ns;
        }
      } else if (ls != KKT_OK) {
        err = ls;
      }
      ras_destroy(m);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(r);
  cudaFree(z);
  if (err != KKT_OK) return err;
  if (best < 0) {
    set_error("ras_autotune: no shape of the subdomain solve fits these subdomains");
    return KKT_ERR_ARG;
  }
  shape_out[0] = best_ch;
  shape_out[1] = best_ns;
  shape_out[2] = kLanes;
  shape_out[3] = 0;
  if (best_ms) *best_ms = best;
  if (cache_path)
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%s\t%d %d %.6f\n", key.c_str(), best_ch, best_ns, best);
      std::fclose(f);
    }
  return KKT_OK;
}
