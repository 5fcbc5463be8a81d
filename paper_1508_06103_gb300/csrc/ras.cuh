// Internal declarations of the Schwarz preconditioner.
#pragma once

#include "internal.cuh"

// slots per point: C row 2*27*2 = 108, G row 2*(27+1) = 56, f row 3*27*2 = 162
constexpr int kSlots = 326;

// A run of at most CH points of one wavefront whose factor values form one
// contiguous block [slot rank][cp] (cp >= n, chosen per precision).
struct Chunk {
  int q0;                      // first point (wavefront order, box-local)
  int n;                       // points
  int cp;                      // row stride of the block
  int box;                     // owning box
  int w;                       // wavefront of the chunk
  int pad_;
  long long off;               // element offset of the block within the box
};

struct GpFactor;   // ILU(1) / point-block ILU(0) factors (iluk.cu)

// One subdomain box (extended set, owned set, storage offsets).
struct BoxDesc {
  int x0, y0, z0, t0;          // origin of the extended box (global node / level)
  int lx, ly, lz, lt;          // extended box extents
  int ox0, ox1, oy0, oy1, oz0, oz1, ot0, ot1;   // owned ranges (global, half open)
  int nlev;                    // wavefronts x + 2y + 4z + 8t
  long long P;                 // points of the extended box
  long long foff;              // offset of the box's chunk blocks (elements)
  long long unit;              // offset of the box's unit row within its factor values (elements)
  long long voff;              // offset of the box's padded local vector (elements)
  long long poff;              // offset into perm / iperm
  long long loff;              // offset into the wavefront pointers
  int cbeg, cend;              // chunk range
  int nown;                    // owned points
  long long ooff;              // offset into the owned-point table
  int kl;                      // exact LU: half-bandwidth of the box matrix
  int prob;                    // problem of the box (a preconditioner over several problems)
  long long aoff;              // exact LU: offset of the box's band (elements)
};

// exact LU: largest half-bandwidth and box size (the solve keeps a box's
// vector in shared memory)
constexpr int kMaxLuBand = 2048;
constexpr int kMaxLuUnknowns = 28672;

struct ras_precond {
  unsigned long long uid = next_handle_uid();
  kkt_problem* prob = nullptr;           // the (first) problem
  // problems of the boxes: one, or several solved together (ras_setup_batch); their
  // unknowns are concatenated in that order, problem k from vec_off[k]
  std::vector<kkt_problem*> probs;
  std::vector<long long> vec_off;        // nprob + 1 offsets
  long long n_total = 0;
  DevProblem* dprobs = nullptr;          // device copies of the problems' DevProblem
  std::vector<DevProblem> dprobs_h;
  int prec = 64;               // factor storage: 64, 32, or 16 (BF16; factorisation and solve in FP32)
  int nbox = 0;
  int ch = 0;                  // points per chunk of the subdomain solve (chosen per preconditioner)
  int cpmax = 0;               // largest chunk row stride
  bool smem_vec = false;       // solve keeps the local vectors in shared memory
  int nstage = 2;              // buffers of the solve's copy ring
  int lanes = 4;               // lanes per point in the solve
  long long fcount = 0;        // factor values
  long long max_pad = 0;       // largest padded local vector (elements)
  long long vcount = 0;        // elements of all padded local vectors (the solve's scratch)
  std::vector<BoxDesc> boxes_h;
  BoxDesc* boxes = nullptr;
  int* perm = nullptr;         // wavefront order -> lexicographic local index
  int* iperm = nullptr;        // lexicographic -> wavefront order
  int* lptr = nullptr;         // wavefront pointers per box (nlev + 1 each)
  Chunk* chunks = nullptr;
  int nchunk = 0;
  int2* gtab = nullptr;        // per point (lexicographic): {3 x global point index, padded offset}
  int2* otab = nullptr;        // per owned point: {3 x global point index, padded offset}
  int* vtab = nullptr;         // per point (wavefront order): padded offset in the box's local vector
  int2* ptab = nullptr;        // per point (wavefront order): {offset of its column in the box's
                               // chunk blocks, row stride of its block}
  void* F = nullptr;           // factor values (FP64, FP32 or BF16, as the solve reads them)
  void* Ffac = nullptr;        // BF16 storage: the FP32 values the factorisation works on
  void* V = nullptr;           // padded local vectors
  int* status = nullptr;
  int local = 0;               // 0: ILU(0) local solves, 1: exact banded LU (FP64)
  double* AB = nullptr;        // exact LU: band factors of all boxes
  long long ab_count = 0;
  int* ipiv = nullptr;         // exact LU: row interchanges (3 per box point)
  int* lu_ju = nullptr;        // exact LU: per box, last column reached by fill (two slots)
  int lu_ctas = 1;             // exact LU: CTAs per box in an elimination step
  TimingLog timing;            // subdomain-solve launches
  TimingLog factor_timing;     // ILU(0) factorisation launches
  BatchWork* bw = nullptr;     // gmres_solve_batch workspace (several problems)
  GpFactor* gp = nullptr;      // local 2 (ILU(1)) or 3 (point-block ILU(0))
};

// shape: NULL, or {chunk points, ring buffers, lanes per point, vector placement
// (1 shared, 2 global)} of the subdomain solve, 0 = chosen automatically.
// Several problems: every problem is split by nsub and all boxes form one list,
// largest first (so the CTAs of a launch finish together as far as they can).
kkt_status ras_create(kkt_problem* const* probs, int nprob, const int nsub[4], int overlap, int local,
                      int factor_prec, const int* shape, ras_precond** out);
// iluk.cu: the pattern-driven local solvers (local 2 and 3)
kkt_status gp_create(ras_precond* m, int local, int prec);
kkt_status gp_factor(ras_precond* m, cudaStream_t s);
kkt_status gp_solve(ras_precond* m, const double* r, double* z, cudaStream_t s, const int* gate);
void gp_destroy(ras_precond* m);
long long gp_factor_count(const ras_precond* m);
kkt_status ras_factor(ras_precond* m, cudaStream_t s);          // enqueue, synchronise, check
kkt_status ras_factor_enqueue(ras_precond* m, cudaStream_t s);  // enqueue only
kkt_status ras_factor_status(ras_precond* m);                   // after the stream completed
// gather and ILU(0) launches of factor32.cu / factor64.cu
kkt_status ras_factor_launch32(ras_precond* m, cudaStream_t s);
kkt_status ras_factor_launch64(ras_precond* m, cudaStream_t s);
kkt_status ras_factor_launch16(ras_precond* m, cudaStream_t s);   // FP32 factorisation, BF16 store
// exact banded LU (lu.cu)
kkt_status ras_lu_factor(ras_precond* m, cudaStream_t s);
kkt_status ras_lu_solve(ras_precond* m, const double* r, double* z, cudaStream_t s, const int* gate);
// the subdomain solve z = M^{-1} r on s; its kernel returns at once while *gate reads 0
// gate_stride: distance (ints) between the gates of consecutive problems; box b
// reads gate[prob(b) * gate_stride]
kkt_status ras_launch(ras_precond* m, const double* r, double* z, cudaStream_t s, const int* gate = nullptr,
                      int gate_stride = 0);
kkt_status ras_check(ras_precond* m);
