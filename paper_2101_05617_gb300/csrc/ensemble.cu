// Batched ensemble: many independent shallow-water members, each on its own
// cubed-sphere grid (n_e, p), advanced together by the multistep EPI method
// (Eq. 25, 30, 34-38) with the adaptive Krylov phi-function solver (Eq. 29).
//
// Every member is an ordinary context: its own grid, tables, Krylov workspace
// and EPI history, and per member the same sequence of operations, the same
// controller (kiops_ctl.h) and the same results as sw_epi_step up to the
// order of floating-point sums.  What is shared:
//
//  * the Krylov iteration.  One persistent kernel launch, captured once in a
//    CUDA graph and replayed, takes one iteration for every member that is
//    building a basis: the imaginary half of the split complex-step JVP
//    (Eq. 28) with the augmented operator, and the window-of-two modified
//    Gram-Schmidt step fused into it (dots in the volume epilogue, then an
//    update + norm pass and a scale + dot pass).  The launch reads the list of
//    members taking part and each member's basis index from device memory, so
//    the same graph serves every iteration.
//    Inside the launch, CTAs take tasks from one atomic counter: the interface
//    tasks of all listed members, then their volume tasks, then the two vector
//    passes.  A task waits (bounded, see wait_count) for its own member's
//    previous phase only.  Tasks are handed out in phase order and every
//    earlier task is held by a CTA that is already running, so every wait
//    ends whatever the number of resident CTAs; members of different sizes
//    share the GPU without any grid-wide barrier.
//  * the exponentials of the small Hessenberg matrices: one launch per matrix
//    product for all members that finished a basis (krylov_device.cuh), and
//  * the host read-backs: one small gather kernel and one copy serve every
//    member that waits for a decision.
//
// Tile shapes (interface points per task, element tiles per task, vector
// entries per task) are per member, and the threads per CTA are per ensemble;
// the autotuner (ens_tune) searches them per (n_e, p) class by timing the
// batched iteration itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "dfr_tangent.cuh"
#include "kiops_ctl.h"
#include "krylov_device.cuh"
#include "swepi_internal.h"

namespace swepi {

namespace {

constexpr int ENS_MAX = 256;                            // members per ensemble
constexpr int ENS_GATHER = 40;                          // doubles read back per member
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // a bounded wait gives up after 2 s
constexpr unsigned int kWaitMaxPolls = 1u << 25;        // ... or after this many polls
constexpr int kBlocks[3] = {128, 256, 512};             // threads per CTA of the batched kernel

// ------------------------------------------------------------------ device data
// Per member: the grid tables and Krylov workspace of its context (fixed), its
// tiles, and the augmented operator of the current KIOPS call.
struct EnsDesc {
  int ns;
  long long nodes, nelem, nfacepts, n;
  const FaceLine* lines;
  const double* fc;
  const double* lf;
  const double* ln;
  double* fb;
  double* V;
  long long ldv;
  double* H;
  int ldh;
  double* cdot;
  int* flags;
  double* vpart;
  double* upart;
  DfrConst dc;
  // tiles
  int face_pts, vol_tiles, vec_len, epb;
  unsigned int n_face, n_vol, n_tiles, pad0;
  // current KIOPS call (uploaded from `tol` to the end)
  double tol, scale, nu;
  const double* b[MAX_NB];
  int p;
  unsigned int n_vec;
};

// Per member, changed by the batched kernel: basis index and phase counters.
struct EnsDyn {
  int j;
  unsigned int face_done, vol_done, upd_done, upd_ticket, scl_ticket, pad0, pad1;
};

// Members of one batched iteration: entry k holds the member and the number
// of tasks of each phase before it; entry `count` holds the totals.
struct EnsEntry {
  int member;
  unsigned int off[4];
};
struct EnsList {
  unsigned int base[5];   // first task of each phase; base[4] = all tasks
  int count;
  int members;            // members of the ensemble (entries of the descriptor array)
  int pad;
  EnsEntry e[ENS_MAX + 1];
};

struct EnsCtl {
  unsigned int next, exited;   // task counter and exit ticket (both back to 0 when a launch ends)
  int error, where;            // a bounded wait gave up: phase | member << 4
  // failure-path test settings (sw_ens_set_wait_test): added to every wait
  // target (0 in normal operation) and the wait's time limit (0 = kWaitLimitNs)
  unsigned int extra, pad;
  unsigned long long limit_ns;
};

struct GatherSrc {
  const double* scal;
  const int* flags;
};

// one exponential of the batch (krylov_device.cuh); N and sq filled after the prep read-back
struct ExpmJob {
  const double* H;
  int ldh, j;
  double tau, tau_happy;
  const int* flags;
  double* ws;
  double* stat;
  double* F;
  int N, sq;
};

// ------------------------------------------------------------------ device code
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 of a task: wait until *ctr >= target.  Every wait here ends by
// construction (see the top of the file); the limit only turns a broken
// invariant into an error status (SW_ETIMEOUT on the host) instead of a hang.
// After a give-up, and once any wait has given up, the task carries on with
// whatever data is there so that the launch still completes.
__device__ void wait_count(const unsigned int* ctr, unsigned int target, EnsCtl* ctl, int where) {
  target += ctl->extra;
  if (ld_acquire(ctr) >= target) return;
  const unsigned long long limit = ctl->limit_ns ? ctl->limit_ns : kWaitLimitNs;
  const unsigned long long t0 = global_ns();
  for (unsigned int it = 1;; ++it) {
    __nanosleep(128);
    if (ld_acquire(ctr) >= target) break;
    if (*(volatile int*)&ctl->error) break;
    if (it >= kWaitMaxPolls || ((it & 255u) == 0 && global_ns() - t0 > limit)) {
      if (atomicCAS(&ctl->error, 0, 1) == 0) ctl->where = where;
      break;
    }
  }
  __threadfence();
}

__device__ __forceinline__ void signal_done(unsigned int* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
  }
}

// the augmented-operator epilogue of iteration j (as kiops_run sets it)
__device__ __forceinline__ AugEpilogue iter_epilogue(const EnsDesc& d, int j) {
  AugEpilogue ep;
  ep.scale = d.scale;
  ep.nu = d.nu;
  ep.p = d.p;
#pragma unroll
  for (int l = 0; l < MAX_NB; ++l) ep.b[l] = d.b[l];
  double* Vi = d.V + (long long)j * d.ldv;
  double* Vn = Vi + d.ldv;
  ep.tail_in = Vi + d.n;
  ep.tail_out = Vn + d.n;
  ep.skip = d.flags;
  ep.dotA = (j >= 1) ? Vi - d.ldv : nullptr;
  ep.dotB = Vi;
  ep.cprev = d.cdot + j;
  ep.h1_out = (j >= 1) ? d.H + (long long)(j - 1) * d.ldh + j : nullptr;
  ep.h2_out = d.H + (long long)j * d.ldh + j;
  ep.dpart = d.vpart;
  ep.dticket = reinterpret_cast<unsigned int*>(d.flags + 9);
  ep.n = d.n;
  return ep;
}

template <int NS, int BLOCK>
__device__ __forceinline__ void face_range(const EnsDesc& d, int j, long long t0, long long t1) {
  TanFaceArgs<double> fa{d.V + (long long)j * d.ldv, nullptr, d.nodes, d.lines, d.fc, d.lf, d.nfacepts, d.fb, nullptr};
  for (long long t = t0 + threadIdx.x; t < t1; t += BLOCK) face_tangent_body<double, NS>(fa, d.dc, t);
}

template <int BLOCK>
__device__ void face_task(const EnsDesc& d, EnsDyn& y, unsigned int local) {
  if (__ldcg(d.flags) == 0) {
    const int j = y.j;
    const long long t0 = (long long)local * d.face_pts;
    const long long t1 = min(t0 + d.face_pts, d.nfacepts);
    switch (d.ns) {
      case 4: face_range<4, BLOCK>(d, j, t0, t1); break;
      case 5: face_range<5, BLOCK>(d, j, t0, t1); break;
      case 6: face_range<6, BLOCK>(d, j, t0, t1); break;
      default: break;
    }
  }
  signal_done(&y.face_done);
}

template <int NS, int BLOCK>
__device__ __forceinline__ void vol_range(const EnsDesc& d, int j, unsigned int local, unsigned char* smem) {
  constexpr int EPB = BLOCK / (NS * NS);
  // the arguments (pointers of iteration j, the augmented operator) in shared
  // memory: read where used instead of held in registers through the body
  __shared__ TanVolArgs<double> sva;
  if (threadIdx.x == 0)
    sva = TanVolArgs<double>{d.V + (long long)j * d.ldv, d.nodes, d.nelem, d.ln, d.fb,
                             d.V + (long long)(j + 1) * d.ldv, iter_epilogue(d, j)};
  __syncthreads();
  const TanVolArgs<double>& va = sva;
  auto& sm = *reinterpret_cast<VolSmem<double, NS, EPB>*>(smem);
  for (int k = 0; k < d.vol_tiles; ++k) {
    const unsigned int tile = local * d.vol_tiles + k;
    if (tile >= d.n_tiles) break;
    if (k > 0) __syncthreads();
    volume_tangent_body<double, NS, EPB, BLOCK>(va, d.dc, tile, d.n_tiles, sm);
  }
}

template <int BLOCK>
__device__ void vol_task(const EnsDesc& d, EnsDyn& y, unsigned int local, EnsCtl* ctl, unsigned char* smem,
                         int member) {
  if (threadIdx.x == 0) wait_count(&y.face_done, d.n_face, ctl, 1 | (member << 4));
  __syncthreads();
  if (__ldcg(d.flags) == 0) {
    const int j = y.j;
    switch (d.ns) {
      case 4: vol_range<4, BLOCK>(d, j, local, smem); break;
      case 5: vol_range<5, BLOCK>(d, j, local, smem); break;
      case 6: vol_range<6, BLOCK>(d, j, local, smem); break;
      default: break;
    }
  }
  signal_done(&y.vol_done);
}

// z -= h1 V_{j-1} + h2 V_j, ||z||_2 -> h_{j+1,j} (and the happy-breakdown flag)
template <int BLOCK>
__device__ void update_task(const EnsDesc& d, EnsDyn& y, unsigned int local, EnsCtl* ctl, int member) {
  if (threadIdx.x == 0) wait_count(&y.vol_done, d.n_vol, ctl, 2 | (member << 4));
  __syncthreads();
  const int j = y.j;
  const bool skip = __ldcg(d.flags) != 0;
  const long long N = d.n + d.p;
  double acc = 0.0;
  if (!skip) {
    double* z = d.V + (long long)(j + 1) * d.ldv;
    const double* VB = d.V + (long long)j * d.ldv;
    const double* VA = (j >= 1) ? VB - d.ldv : nullptr;
    const double h1 = VA ? __ldcg(d.H + (long long)(j - 1) * d.ldh + j) : 0.0;
    const double h2 = __ldcg(d.H + (long long)j * d.ldh + j);
    const long long i0 = (long long)local * d.vec_len, i1 = min(i0 + d.vec_len, N);
    acc = mgs_update_range(z, VA, VB, h1, h2, i0 + threadIdx.x, i1, BLOCK);
  }
  const double b = block_sum<BLOCK>(acc);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    d.upart[local] = b;
    __threadfence();
    last = atomicAdd(&y.upd_ticket, 1u) == d.n_vec - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (unsigned int k = threadIdx.x; k < d.n_vec; k += BLOCK) s += __ldcg(d.upart + k);
    s = block_sum<BLOCK>(s);
    if (threadIdx.x == 0) {
      if (!skip) {
        const double r = sqrt(s);
        d.H[(long long)(j + 1) * d.ldh + j] = r;
        if (r < d.tol) {
          d.flags[1] = j + 1;
          d.flags[0] = 1;
        }
      }
      y.upd_ticket = 0u;
    }
  }
  signal_done(&y.upd_done);
}

// V_{j+1} = z / h_{j+1,j}, V_{j+1} . V_j -> cdot[j+1]; the member's last task
// resets the phase counters and advances its basis index
template <int BLOCK>
__device__ void scale_task(const EnsDesc& d, EnsDyn& y, unsigned int local, EnsCtl* ctl, int member) {
  if (threadIdx.x == 0) wait_count(&y.upd_done, d.n_vec, ctl, 3 | (member << 4));
  __syncthreads();
  const int j = y.j;
  const bool skip = __ldcg(d.flags) != 0;
  const long long N = d.n + d.p;
  double acc = 0.0;
  if (!skip) {
    double* z = d.V + (long long)(j + 1) * d.ldv;
    const double* VB = d.V + (long long)j * d.ldv;
    const double r = 1.0 / __ldcg(d.H + (long long)(j + 1) * d.ldh + j);
    const long long i0 = (long long)local * d.vec_len, i1 = min(i0 + d.vec_len, N);
    acc = scale_dot_range(z, VB, r, i0 + threadIdx.x, i1, BLOCK);
  }
  const double b = block_sum<BLOCK>(acc);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    d.upart[local] = b;
    __threadfence();
    last = atomicAdd(&y.scl_ticket, 1u) == d.n_vec - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (unsigned int k = threadIdx.x; k < d.n_vec; k += BLOCK) s += __ldcg(d.upart + k);
  s = block_sum<BLOCK>(s);
  if (threadIdx.x == 0) {
    if (!skip) d.cdot[j + 1] = s;
    y.face_done = 0u;
    y.vol_done = 0u;
    y.upd_done = 0u;
    y.scl_ticket = 0u;
    y.j = j + 1;
    __threadfence();
  }
}

template <int BLOCK>
struct VolBytes {
  static constexpr size_t a = sizeof(VolSmem<double, 4, BLOCK / 16>);
  static constexpr size_t b = sizeof(VolSmem<double, 5, BLOCK / 25>);
  static constexpr size_t c = sizeof(VolSmem<double, 6, BLOCK / 36>);
  static constexpr size_t value = (a > b ? (a > c ? a : c) : (b > c ? b : c));
};

// checked build: the task a CTA decoded names a listed member of the
// ensemble, lies inside that member's tasks of its phase, and the member's
// basis index leaves room for V_{j+1}
__device__ __forceinline__ bool ens_task_ok(const EnsList& L, int lo, int ph, unsigned int rel,
                                            const EnsDesc* desc, const EnsDyn* dyn) {
  if (lo < 0 || lo >= L.count || ph < 0 || ph > 3) return false;
  const int m = L.e[lo].member;
  if (m < 0 || m >= L.members || rel < L.e[lo].off[ph]) return false;
  const EnsDesc& d = desc[m];
  const unsigned int local = rel - L.e[lo].off[ph];
  const unsigned int n = ph == 0 ? d.n_face : (ph == 1 ? d.n_vol : d.n_vec);
  const int j = dyn[m].j;
  return local < n && j >= 0 && j + 1 <= d.ldh - 2;
}

// one Krylov iteration of every listed member (persistent, graph-captured);
// 64 registers per thread at most (1024 threads per SM), as the single-grid
// volume kernel
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) ens_iter_kernel(const EnsDesc* __restrict__ desc, EnsDyn* __restrict__ dyn,
                                                         const EnsList* __restrict__ list, EnsCtl* ctl) {
  __shared__ unsigned int s_task;
  __shared__ __align__(16) unsigned char s_vol[VolBytes<BLOCK>::value];
  const unsigned int total = list->base[4];
  const int count = list->count;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_task = atomicAdd(&ctl->next, 1u);
    __syncthreads();
    const unsigned int task = s_task;
    if (task >= total) break;
    int ph = 0;
    while (ph < 3 && task >= list->base[ph + 1]) ++ph;
    const unsigned int rel = task - list->base[ph];
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (list->e[mid].off[ph] <= rel) lo = mid;
      else hi = mid - 1;
    }
    if (kChecked) {   // checked build: thread 0 decides for the CTA; a bad task is skipped
      __shared__ int s_ok;
      if (threadIdx.x == 0) {
        s_ok = ens_task_ok(*list, lo, ph, rel, desc, dyn);
        if (!s_ok) check_fail(CHK_ENS_TASK);
      }
      __syncthreads();
      if (!s_ok) continue;
    }
    const int m = list->e[lo].member;
    const unsigned int local = rel - list->e[lo].off[ph];
    const EnsDesc& d = desc[m];
    EnsDyn& y = dyn[m];
    if (ph == 0) face_task<BLOCK>(d, y, local);
    else if (ph == 1) vol_task<BLOCK>(d, y, local, ctl, s_vol, m);
    else if (ph == 2) update_task<BLOCK>(d, y, local, ctl, m);
    else scale_task<BLOCK>(d, y, local, ctl, m);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl->exited, 1u) == gridDim.x - 1) {
      ctl->next = 0u;
      ctl->exited = 0u;
      __threadfence();
    }
  }
}

// ---- batched exponential (one CTA per member, then one launch per product)
__global__ void ens_expm_prep_kernel(const ExpmJob* __restrict__ jobs) {
  const ExpmJob& jb = jobs[blockIdx.x];
  expm_prep_body(jb.H, jb.ldh, jb.j, jb.tau, jb.tau_happy, jb.flags, jb.ws, jb.stat);
}

__global__ void __launch_bounds__(64) ens_expm_gemm_kernel(const ExpmJob* __restrict__ jobs, int sc, int sa, int sb,
                                                           MatEpi e, int scaling) {
  const ExpmJob& jb = jobs[blockIdx.z];
  const int r = blockIdx.y * 8 + threadIdx.y, c = blockIdx.x * 8 + threadIdx.x;
  if (r >= jb.N || c >= jb.N) return;
  if (scaling) e.alpha = ldexp(1.0, -jb.sq);
  expm_gemm_entry(jb.ws, jb.N, sc, sa, sb, e, r, c);
}

__global__ void __launch_bounds__(64) ens_expm_square_kernel(const ExpmJob* __restrict__ jobs, int q) {
  const ExpmJob& jb = jobs[blockIdx.z];
  const int r = blockIdx.y * 8 + threadIdx.y, c = blockIdx.x * 8 + threadIdx.x;
  if (q >= jb.sq || r >= jb.N || c >= jb.N) return;
  const MatEpi none{0, 0, 0, 0, -1, -1, -1, 1.0};
  const int src = expm_square_src(q);
  expm_gemm_entry(jb.ws, jb.N, expm_square_dst(q), src, src, none, r, c);
}

__global__ void ens_expm_finish_kernel(const ExpmJob* __restrict__ jobs) {
  const ExpmJob& jb = jobs[blockIdx.y];
  const long long NN = (long long)jb.N * jb.N;
  const double* P = jb.ws + expm_result_slot(jb.sq) * NN;
  for (long long i = threadIdx.x + (long long)blockIdx.x * blockDim.x; i < NN; i += (long long)blockDim.x * gridDim.x)
    expm_finish_entry(P, jb.N, jb.F, jb.ldh, jb.stat, i);
}

// scalars and flags of every member, and the wait status, into one buffer
__global__ void ens_gather_kernel(const GatherSrc* __restrict__ src, int count, const EnsCtl* ctl, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count * ENS_GATHER; i += blockDim.x * gridDim.x) {
    const int m = i / ENS_GATHER, k = i % ENS_GATHER;
    double v = 0.0;
    if (k < 32) v = src[m].scal[k];
    else if (k < 36) v = (double)src[m].flags[k - 32];
    out[i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[count * ENS_GATHER] = (double)ctl->error;
    out[count * ENS_GATHER + 1] = (double)ctl->where;
  }
}

}  // namespace

// ------------------------------------------------------------------ host side
namespace {

enum CallState { CS_IDLE = 0, CS_SETUP1, CS_SETUP2, CS_ITER, CS_PREP, CS_EVAL, CS_DONE };
enum WaitState { W_NONE = 0, W_READ, W_ITER, W_PREP, W_EVAL, W_DONE };

struct Member {
  Ctx* c = nullptr;
  int klass = 0;
  sw_ens_tiles tiles{};
  // EPI run
  int order = 0;
  double dt = 0.0;
  double* q = nullptr;
  int steps_total = 0, steps_done = 0;
  int kind = 0, sub = 0;   // 0 EPI2 step, 1 start-up substeps, 2 multistep
  double h = 0.0;          // step of the current EPI2 (sub)step
  sw_kiops_stats acc{};
  // KIOPS call
  int cst = CS_IDLE, wait = W_NONE;
  KiopsController K;
  sw_kiops_opts o{};
  int p = 1;
  double nu = 1.0, mu = 1.0, normb = 0.0, dtc = 0.0;
  const double* bk[MAX_NB + 1] = {};
  double* w = nullptr;
  float feat[16] = {};
  int m_cur = 0, j_dev = -1, ne_expm = 0, sq = 0;
};

}  // namespace

struct Ens {
  int device = 0;
  int count = 0;
  // a run that ended with an error (e.g. a wait that gave up) can leave the
  // members' phase counters part-way: the next run clears them first
  bool dyn_stale = false;
  std::vector<Member> mem;
  std::vector<EnsDesc> hdesc;
  std::vector<EnsDyn> hdyn;
  EnsDesc* d_desc = nullptr;
  EnsDyn* d_dyn = nullptr;
  EnsList* d_list = nullptr;
  EnsCtl* d_ctl = nullptr;
  GatherSrc* d_gsrc = nullptr;
  double* d_gather = nullptr;
  double* h_gather = nullptr;
  ExpmJob* d_jobs = nullptr;
  double* d_upart = nullptr;
  long long upart_stride = 0;
  // pinned staging ring for host-to-device uploads (reset at every full synchronisation)
  unsigned char* h_ring = nullptr;
  size_t ring_cap = 0, ring_off = 0;
  int block = 256;
  int ctas[3] = {0, 0, 0};
  cudaGraph_t graph[3] = {};
  cudaGraphExec_t gexec[3] = {};
  cudaStream_t cap_stream = nullptr;
  EnsList hlist{};
  std::vector<int> last_ids;
  bool list_dirty = true;
  int last_block = -1;
  double theta = 0.5;
  sw_ens_stats st{};
  // per-member streams: a member's own kernels (RHS, linearisation, remainders,
  // norms, combinations) overlap with other members'; the shared stream waits
  // on a member's stream (event) before any batched work that touches it
  std::vector<cudaStream_t> mstream;
  std::vector<cudaEvent_t> mevent;
  std::vector<char> dirty;
  cudaEvent_t start_event = nullptr;   // member streams wait for the caller's stream at a run's start
  // event timing of the batched iterations (sw_ens_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
  size_t ev_used = 0;
};

}  // namespace swepi

struct sw_ens : public swepi::Ens {};

namespace swepi {
namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? SW_OK : SW_ECUDA; }

int block_index(int block) {
  for (int i = 0; i < 3; ++i)
    if (kBlocks[i] == block) return i;
  return -1;
}

sw_ens_tiles default_tiles(int block) { return sw_ens_tiles{2 * block, 1, 16 * block}; }

bool tiles_valid(const sw_ens_tiles& t) {
  return t.face_pts >= 32 && t.face_pts <= (1 << 20) && t.vol_tiles >= 1 && t.vol_tiles <= 64 && t.vec_len >= 128 &&
         t.vec_len <= (1 << 24);
}

// pinned staging of an upload; the copy is issued on s
int upload(Ens& e, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  const size_t need = (bytes + 255) & ~size_t(255);
  if (need > e.ring_cap) return SW_EINVAL;
  if (e.ring_off + need > e.ring_cap) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return SW_ECUDA;
    e.ring_off = 0;
  }
  unsigned char* h = e.h_ring + e.ring_off;
  std::memcpy(h, src, bytes);
  e.ring_off += need;
  return cuda_rc(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, s));
}

// task counts of member m for the current block / tiles / p
void set_counts(Ens& e, int m) {
  EnsDesc& d = e.hdesc[m];
  const sw_ens_tiles& t = e.mem[m].tiles;
  d.epb = e.block / (d.ns * d.ns);
  d.face_pts = t.face_pts;
  d.vol_tiles = t.vol_tiles;
  d.vec_len = t.vec_len;
  d.n_face = (unsigned int)((d.nfacepts + t.face_pts - 1) / t.face_pts);
  d.n_tiles = (unsigned int)((d.nelem + d.epb - 1) / d.epb);
  d.n_vol = (d.n_tiles + t.vol_tiles - 1) / t.vol_tiles;
  d.n_vec = (unsigned int)((d.n + d.p + t.vec_len - 1) / t.vec_len);
}

int upload_desc(Ens& e, int m, cudaStream_t s) {
  set_counts(e, m);
  e.list_dirty = true;
  return upload(e, e.d_desc + m, &e.hdesc[m], sizeof(EnsDesc), s);
}

int upload_j(Ens& e, int m, int j, cudaStream_t s) {
  e.hdyn[m].j = j;
  e.mem[m].j_dev = j;
  return upload(e, &e.d_dyn[m].j, &e.hdyn[m].j, sizeof(int), s);
}

// the stream of member m's own kernels (marks it as having unjoined work)
cudaStream_t member_stream(Ens& e, int m) {
  e.dirty[m] = 1;
  return e.mstream[m];
}

// make the shared stream s wait for member m's issued work
int join_member(Ens& e, int m, cudaStream_t s) {
  if (!e.dirty[m]) return SW_OK;
  e.dirty[m] = 0;
  if (cudaEventRecord(e.mevent[m], e.mstream[m]) != cudaSuccess) return SW_ECUDA;
  return cuda_rc(cudaStreamWaitEvent(s, e.mevent[m], 0));
}

int join_all(Ens& e, cudaStream_t s) {
  int rc;
  for (int m = 0; m < e.count; ++m)
    if ((rc = join_member(e, m, s))) return rc;
  return SW_OK;
}

template <int BLOCK>
int capture_block(Ens& e, int bi) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ens_iter_kernel<BLOCK>, BLOCK, 0) != cudaSuccess || nb < 1)
    return SW_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e.device) != cudaSuccess) return SW_ECUDA;
  e.ctas[bi] = nb * sms;
  if (cudaStreamBeginCapture(e.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SW_ECUDA;
  ens_iter_kernel<BLOCK><<<e.ctas[bi], BLOCK, 0, e.cap_stream>>>(e.d_desc, e.d_dyn, e.d_list, e.d_ctl);
  cudaError_t le = cudaGetLastError();
  cudaError_t ce = cudaStreamEndCapture(e.cap_stream, &e.graph[bi]);
  if (le != cudaSuccess || ce != cudaSuccess) return SW_ECUDA;
  if (cudaGraphInstantiate(&e.gexec[bi], e.graph[bi], 0) != cudaSuccess) return SW_ECUDA;
  return SW_OK;
}

int ensure_graph(Ens& e, int block) {
  const int bi = block_index(block);
  if (bi < 0) return SW_EINVAL;
  if (e.gexec[bi]) return SW_OK;
  switch (block) {
    case 128: return capture_block<128>(e, bi);
    case 256: return capture_block<256>(e, bi);
    default: return capture_block<512>(e, bi);
  }
}

// one batched Krylov iteration of the members in `ids` (graph replay)
int launch_iteration(Ens& e, const std::vector<int>& ids, cudaStream_t s) {
  if (ids.empty()) return SW_OK;
  for (int m : ids) {
    int rc = join_member(e, m, s);
    if (rc) return rc;
  }
  if (ids != e.last_ids || e.list_dirty || e.last_block != e.block) {
    EnsList& L = e.hlist;
    L.count = (int)ids.size();
    L.members = e.count;
    unsigned int tot[4] = {0, 0, 0, 0};
    for (int k = 0; k < L.count; ++k) {
      const EnsDesc& d = e.hdesc[ids[k]];
      L.e[k].member = ids[k];
      for (int ph = 0; ph < 4; ++ph) L.e[k].off[ph] = tot[ph];
      tot[0] += d.n_face;
      tot[1] += d.n_vol;
      tot[2] += d.n_vec;
      tot[3] += d.n_vec;
    }
    L.e[L.count].member = -1;
    for (int ph = 0; ph < 4; ++ph) L.e[L.count].off[ph] = tot[ph];
    L.base[0] = 0;
    for (int ph = 0; ph < 4; ++ph) L.base[ph + 1] = L.base[ph] + tot[ph];
    const size_t bytes = offsetof(EnsList, e) + sizeof(EnsEntry) * (L.count + 1);
    int rc = upload(e, e.d_list, &L, bytes, s);
    if (rc) return rc;
    e.last_ids = ids;
    e.list_dirty = false;
    e.last_block = e.block;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (e.prof) {
    while (e.ev_pool.size() < e.ev_used + 2) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) return SW_ECUDA;
      e.ev_pool.push_back(ev);
    }
    a = e.ev_pool[e.ev_used++];
    b = e.ev_pool[e.ev_used++];
    cudaEventRecord(a, s);
  }
  if (cudaGraphLaunch(e.gexec[block_index(e.block)], s) != cudaSuccess) return SW_ECUDA;
  if (e.prof) {
    cudaEventRecord(b, s);
    e.ev_pending.push_back({a, b});
  }
  e.st.ticks++;
  e.st.launches++;
  return SW_OK;
}

// after a full synchronisation: add the timed iterations to the statistics
void drain_events(Ens& e) {
  for (auto& pr : e.ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) e.st.iter_ms += ms;
  }
  e.ev_pending.clear();
  e.ev_used = 0;
}

// one read-back of every member's scalars and flags (a full synchronisation)
int gather(Ens& e, cudaStream_t s) {
  int rc = join_all(e, s);
  if (rc) return rc;
  ens_gather_kernel<<<(e.count * ENS_GATHER + 255) / 256, 256, 0, s>>>(e.d_gsrc, e.count, e.d_ctl, e.d_gather);
  e.st.launches++;
  if (cudaGetLastError() != cudaSuccess) return SW_ECUDA;
  if (cudaMemcpyAsync(e.h_gather, e.d_gather, sizeof(double) * (e.count * ENS_GATHER + 2), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess)
    return SW_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SW_ECUDA;
  e.ring_off = 0;
  drain_events(e);
  e.st.reads++;
  if (e.h_gather[e.count * ENS_GATHER] != 0.0) return SW_ETIMEOUT;
  return SW_OK;
}

// ---------------------------------------------------------------- KIOPS call
int call_start(Ens& e, int m, double dt, int nb, const double* const* b, double* w, const sw_kiops_opts& o0,
               cudaStream_t s) {
  Member& M = e.mem[m];
  Ctx& c = *M.c;
  const cudaStream_t ms = member_stream(e, m);   // s: the shared stream (uploads)
  M.o = o0;
  if (c.m_warm > 0) M.o.m_init = c.m_warm;   // warm start from the previous call (as phi_call)
  const long long n = c.n;
  int p = nb - 1;
  for (int k = 0; k <= MAX_NB; ++k) M.bk[k] = (k < nb) ? b[k] : nullptr;
  if (p == 0) {
    p = 1;
    M.bk[1] = nullptr;
  }
  M.p = p;
  M.dtc = dt;
  M.w = w;
  int rc;
  for (int k = 1; k <= p; ++k) {
    if (M.bk[k]) {
      if ((rc = launch_norm1(c, M.bk[k], n, c.d_scal + S_NORMB + k, ms))) return rc;
    } else if (cudaMemsetAsync(c.d_scal + S_NORMB + k, 0, sizeof(double), ms) != cudaSuccess) {
      return SW_ECUDA;
    }
  }
  if (M.bk[0]) {
    if (cudaMemcpyAsync(c.d_X, M.bk[0], sizeof(double) * n, cudaMemcpyDeviceToDevice, ms) != cudaSuccess)
      return SW_ECUDA;
  } else if (cudaMemsetAsync(c.d_X, 0, sizeof(double) * n, ms) != cudaSuccess) {
    return SW_ECUDA;
  }
  M.cst = CS_SETUP1;
  M.wait = W_READ;
  return SW_OK;
}

int epi_after_call(Ens& e, int m, const sw_kiops_opts& o, cudaStream_t s);

int attempt(Ens& e, int m, const sw_kiops_opts& o, cudaStream_t s) {
  Member& M = e.mem[m];
  Ctx& c = *M.c;
  const cudaStream_t ms = member_stream(e, m);   // s: the shared stream (uploads)
  KiopsController& K = M.K;
  int rc;
  if (K.done()) {
    if (cudaMemcpyAsync(M.w, c.d_X, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, ms) != cudaSuccess)
      return SW_ECUDA;
    sw_kiops_stats st{};
    kiops_finish_call(c, K, M.feat, M.o, &st);
    c.m_warm = st.m_final;
    add_stats(&M.acc, st);
    M.cst = CS_DONE;
    return epi_after_call(e, m, o, s);
  }
  const long long N = c.n + M.p;
  const int j = K.j;
  M.m_cur = K.m;
  if (j == 0) {
    if ((rc = launch_norm2(c, c.d_X, N, c.d_scal + S_BETA, 0.0, nullptr, 0, nullptr, ms))) return rc;
    if ((rc = launch_scale_inv(c, c.d_V, c.d_X, c.d_scal + S_BETA, N, nullptr, ms))) return rc;
    if (cudaMemsetAsync(c.d_flags, 0, sizeof(int) * 2, ms) != cudaSuccess) return SW_ECUDA;
    if (cudaMemsetAsync(c.d_H, 0, sizeof(double) * c.ldh * c.ldh, ms) != cudaSuccess) return SW_ECUDA;
  }
  if (j < M.m_cur) {
    if (M.j_dev != j && (rc = upload_j(e, m, j, s))) return rc;
    M.cst = CS_ITER;
    M.wait = W_ITER;
  } else {
    M.cst = CS_PREP;
    M.wait = W_PREP;
  }
  return SW_OK;
}

// the read-back of member m is in g (ENS_GATHER doubles)
int on_read(Ens& e, int m, const double* g, const sw_kiops_opts& o, std::vector<int>& evals, cudaStream_t s) {
  Member& M = e.mem[m];
  Ctx& c = *M.c;
  const cudaStream_t ms = member_stream(e, m);   // s: the shared stream (uploads)
  int rc;
  switch (M.cst) {
    case CS_SETUP1: {
      double normb = 0.0;
      for (int k = 1; k <= M.p; ++k) normb = std::max(normb, g[S_NORMB + k]);
      if (!std::isfinite(normb)) return SW_ENONFINITE;
      M.normb = normb;
      M.nu = 1.0;
      M.mu = 1.0;
      if (normb > 0) {
        const int ex = (int)std::ceil(std::log2(normb));
        M.nu = std::ldexp(1.0, -ex);
        M.mu = std::ldexp(1.0, ex);
      }
      double tail[MAX_NB] = {};
      tail[M.p - 1] = M.mu;
      if ((rc = launch_set_tail(c, c.d_X, c.n, M.p, tail, ms))) return rc;
      if ((rc = launch_norm2(c, c.d_X, c.n + M.p, c.d_scal + S_BETA0, 0.0, nullptr, 0, nullptr, ms))) return rc;
      M.cst = CS_SETUP2;
      M.wait = W_READ;
      return SW_OK;
    }
    case CS_SETUP2: {
      const double beta0 = g[S_BETA0];
      if (!std::isfinite(beta0)) return SW_ENONFINITE;
      kiops_features(c, M.normb, beta0, M.dtc, M.p, M.feat);
      const double tau_end = 1.0;
      const double tau = (M.o.tau_init > 0) ? std::min(M.o.tau_init, tau_end) : tau_end;
      const int m0 = std::min(std::max(M.o.m_init, M.o.m_min), M.o.m_max);
      M.K = KiopsController();
      M.K.start(tau_end, M.o.tol, beta0, M.o, tau, m0);
      EnsDesc& d = e.hdesc[m];
      d.tol = M.o.tol;
      d.scale = M.dtc;
      d.nu = M.nu;
      d.p = M.p;
      for (int l = 0; l < MAX_NB; ++l) d.b[l] = (l < M.p) ? M.bk[M.p - l] : nullptr;
      if ((rc = upload_desc(e, m, s))) return rc;
      return attempt(e, m, o, s);
    }
    case CS_PREP: {
      const int Ne = (int)g[S_STAT + 1] + 1;
      const double norm1 = g[S_STAT + 5];
      if (Ne < 2 || Ne > MAX_EXPM || !std::isfinite(norm1)) return SW_EINVAL;
      const int sq = expm_squarings(norm1);
      if (sq < 0) return SW_ENONFINITE;
      M.ne_expm = Ne;
      M.sq = sq;
      M.cst = CS_EVAL;
      M.wait = W_EVAL;
      evals.push_back(m);
      return SW_OK;
    }
    case CS_EVAL: {
      KiopsController& K = M.K;
      const bool happy = g[32] != 0.0;
      if ((rc = K.decide(happy, happy ? (int)g[33] : M.m_cur, g[S_BETA], g[S_STAT + 4], g[S_STAT + 0]))) return rc;
      if (K.accept && (rc = launch_combine(c, K.j_used, c.n, ms))) return rc;
      if ((rc = K.finish(kMaxSubsteps, kMaxRejects))) return rc;
      if (K.accept) {
        double tv[MAX_NB];
        K.tail(M.p, M.mu, tv);
        if ((rc = launch_set_tail(c, c.d_X, c.n, M.p, tv, ms))) return rc;
      }
      return attempt(e, m, o, s);
    }
    default: return SW_EINVAL;
  }
}

// ---------------------------------------------------------------- EPI driver (as sw_epi_step)
int epi_begin_step(Ens& e, int m, const sw_kiops_opts& o, cudaStream_t s);

// one exponential-Euler (sub)step (Eq. 25) of size h: b_1 = h F(q)
int epi2_start(Ens& e, int m, double h, const sw_kiops_opts& o, cudaStream_t s) {
  Member& M = e.mem[m];
  Ctx& c = *M.c;
  const cudaStream_t ms = member_stream(e, m);   // s: the shared stream (uploads)
  int rc;
  M.h = h;
  const double* xs[1] = {c.d_Fn};
  double cf[1] = {h};
  if ((rc = launch_lincomb(c, c.d_b[0], c.n, 1, xs, cf, ms))) return rc;
  if ((rc = launch_linearize(c, M.q, ms))) return rc;
  const double* b[2] = {nullptr, c.d_b[0]};
  return call_start(e, m, h, 2, b, c.d_tmp, o, s);
}

int epi_begin_step(Ens& e, int m, const sw_kiops_opts& o, cudaStream_t s) {
  Member& M = e.mem[m];
  Ctx& c = *M.c;
  const cudaStream_t ms = member_stream(e, m);   // s: the shared stream (uploads)
  const long long n = c.n;
  int rc;
  c.epi_order = M.order;
  c.epi_stage = 0;
  if ((rc = launch_rhs(c, M.q, c.d_Fn, ms))) return rc;
  if (M.order == 2) {
    M.kind = 0;
    return epi2_start(e, m, M.dt, o, s);
  }
  const Coefs* A = coefs_for(M.order);
  if (c.hist_count < A->P) {
    // start-up: EPI2 with smaller substeps (Sec. 4)
    if ((rc = push_history(c, M.q, c.d_Fn, ms))) return rc;
    c.epi_stage = 1;
    M.kind = 1;
    M.sub = 0;
    return epi2_start(e, m, M.dt / EPI_STARTUP_SUBSTEPS, o, s);
  }
  M.kind = 2;
  // remainders R(q_{n-i}) = F(q_{n-i}) - F_n - J_n (q_{n-i} - q_n)  (Eq. 33)
  if ((rc = launch_linearize(c, M.q, ms))) return rc;
  for (int i = 1; i <= A->P; ++i) {
    const int slot = hist_slot(c, i);
    const double* d1[2] = {c.d_hq[slot], M.q};
    double c1[2] = {1.0, -1.0};
    if ((rc = launch_lincomb(c, c.d_tmp, n, 2, d1, c1, ms))) return rc;
    AugEpilogue ep;
    if ((rc = launch_jvp_lin(c, c.d_tmp, c.d_tmp2, ep, ms, false))) return rc;
    const double* d2[3] = {c.d_hF[slot], c.d_Fn, c.d_tmp2};
    double c2[3] = {1.0, -1.0, -1.0};
    if ((rc = launch_lincomb(c, c.d_R[i - 1], n, 3, d2, c2, ms))) return rc;
  }
  // b_1 = dt F_n + v_1, b_m = v_m with v_m = sum_i alpha_{m,i} dt R_i  (Eq. 34-35)
  for (int k = 0; k < A->M; ++k) {
    const double* xs[MAX_HIST + 1];
    double cf[MAX_HIST + 1];
    int t = 0;
    if (k == 0) {
      xs[t] = c.d_Fn;
      cf[t] = M.dt;
      ++t;
    }
    for (int i = 0; i < A->P; ++i) {
      xs[t] = c.d_R[i];
      cf[t] = A->a[k][i] * M.dt;
      ++t;
    }
    if ((rc = launch_lincomb(c, c.d_b[k], n, t, xs, cf, ms))) return rc;
  }
  const double* b[MAX_NB] = {nullptr};
  for (int k = 0; k < A->M; ++k) b[k + 1] = c.d_b[k];
  return call_start(e, m, M.dt, A->M + 1, b, c.d_tmp, o, s);
}

int epi_after_call(Ens& e, int m, const sw_kiops_opts& o, cudaStream_t s) {
  Member& M = e.mem[m];
  Ctx& c = *M.c;
  const cudaStream_t ms = member_stream(e, m);   // s: the shared stream (uploads)
  int rc;
  const double* ys[2] = {M.q, c.d_tmp};
  double one[2] = {1.0, 1.0};
  if (M.kind == 2 && (rc = push_history(c, M.q, c.d_Fn, ms))) return rc;
  if ((rc = launch_lincomb(c, M.q, c.n, 2, ys, one, ms))) return rc;
  if (M.kind == 1 && ++M.sub < EPI_STARTUP_SUBSTEPS) {
    if ((rc = launch_rhs(c, M.q, c.d_Fn, ms))) return rc;
    return epi2_start(e, m, M.h, o, s);
  }
  if (M.kind == 1) c.epi_stage = 0;
  M.steps_done++;
  if (M.steps_done < M.steps_total) return epi_begin_step(e, m, o, s);
  M.cst = CS_IDLE;
  M.wait = W_DONE;
  return SW_OK;
}

// ---------------------------------------------------------------- batched exponential
int launch_prep_batch(Ens& e, std::vector<ExpmJob>& jobs, std::vector<int>& ids, cudaStream_t s) {
  jobs.clear();
  ids.clear();
  for (int m = 0; m < e.count; ++m) {
    Member& M = e.mem[m];
    if (M.wait != W_PREP) continue;
    Ctx& c = *M.c;
    if (M.m_cur + 1 > MAX_EXPM) return SW_EINVAL;
    int rc = join_member(e, m, s);
    if (rc) return rc;
    ExpmJob jb{c.d_H, c.ldh, M.m_cur, M.K.tau, M.K.tau_end - M.K.tau_now, c.d_flags, c.d_expm_ws, c.d_scal + S_STAT,
               c.d_F, 0, 0};
    jobs.push_back(jb);
    ids.push_back(m);
    M.wait = W_READ;
  }
  if (jobs.empty()) return SW_OK;
  int rc = upload(e, e.d_jobs, jobs.data(), sizeof(ExpmJob) * jobs.size(), s);
  if (rc) return rc;
  ens_expm_prep_kernel<<<(unsigned)jobs.size(), 256, 0, s>>>(e.d_jobs);
  e.st.launches++;
  return cuda_rc(cudaGetLastError());
}

int launch_eval_batch(Ens& e, const std::vector<int>& evals, cudaStream_t s) {
  if (evals.empty()) return SW_OK;
  std::vector<ExpmJob> jobs;
  int maxN = 0, maxsq = 0;
  for (int m : evals) {
    Member& M = e.mem[m];
    Ctx& c = *M.c;
    int rcj = join_member(e, m, s);
    if (rcj) return rcj;
    ExpmJob jb{c.d_H, c.ldh, M.m_cur, 0.0, 0.0, c.d_flags, c.d_expm_ws, c.d_scal + S_STAT, c.d_F, M.ne_expm, M.sq};
    jobs.push_back(jb);
    maxN = std::max(maxN, M.ne_expm);
    maxsq = std::max(maxsq, M.sq);
    M.wait = W_READ;
  }
  int rc = upload(e, e.d_jobs, jobs.data(), sizeof(ExpmJob) * jobs.size(), s);
  if (rc) return rc;
  const unsigned nj = (unsigned)jobs.size();
  const dim3 blk(8, 8), grd((maxN + 7) / 8, (maxN + 7) / 8, nj);
  ExpmProduct pr[8];
  expm_products(0, pr);
  for (int k = 0; k < 8; ++k)
    ens_expm_gemm_kernel<<<grd, blk, 0, s>>>(e.d_jobs, pr[k].c, pr[k].a, pr[k].b, pr[k].e, k == 0 ? 1 : 0);
  for (int q = 0; q < maxsq; ++q) ens_expm_square_kernel<<<grd, blk, 0, s>>>(e.d_jobs, q);
  const long long NN = (long long)maxN * maxN;
  ens_expm_finish_kernel<<<dim3((unsigned)((NN + 255) / 256), nj), 256, 0, s>>>(e.d_jobs);
  e.st.launches += 9 + maxsq;
  e.st.expm_batches++;
  return cuda_rc(cudaGetLastError());
}

long long member_launches(const Ens& e) {
  long long t = 0;
  for (const Member& M : e.mem) t += M.c->launches;
  return t;
}

}  // namespace

// ---------------------------------------------------------------- run
int ens_run(Ens& e, int steps, const int* orders, const double* dts, double* const* q, const sw_kiops_opts& o,
            sw_kiops_stats* stats, cudaStream_t s) {
  int rc;
  if ((rc = ensure_graph(e, e.block))) return rc;
  e.st = sw_ens_stats{};
  const long long l0 = member_launches(e);
  for (int m = 0; m < e.count; ++m) {
    Member& M = e.mem[m];
    Ctx& c = *M.c;
    if ((rc = ensure_epi(c)) || (rc = ensure_krylov(c, o.m_max))) return rc;
    // the Krylov workspace may have moved
    EnsDesc& d = e.hdesc[m];
    d.V = c.d_V;
    d.ldv = c.ldv;
    d.H = c.d_H;
    d.ldh = c.ldh;
    d.cdot = c.d_cdot;
    d.vpart = c.d_vpart;
    d.flags = c.d_flags;
    M.order = orders[m];
    M.dt = dts[m];
    M.q = q[m];
    M.steps_total = steps;
    M.steps_done = 0;
    M.acc = sw_kiops_stats{};
    M.cst = CS_IDLE;
    M.wait = W_DONE;
    M.j_dev = -1;
  }
  // the caller's earlier work on s (e.g. the initial states) comes first
  if (cudaEventRecord(e.start_event, s) != cudaSuccess) return SW_ECUDA;
  for (int m = 0; m < e.count; ++m)
    if (cudaStreamWaitEvent(e.mstream[m], e.start_event, 0) != cudaSuccess) return SW_ECUDA;
  for (int m = 0; m < e.count; ++m) {
    if (steps == 0) break;
    // the lin tables are allocated by the first linearisation: start each member, then refresh its tables
    if ((rc = epi_begin_step(e, m, o, s))) return rc;
  }
  for (int m = 0; m < e.count; ++m) {
    Ctx& c = *e.mem[m].c;
    EnsDesc& d = e.hdesc[m];
    d.lf = c.d_lin_face;
    d.ln = c.d_lin_node;
    if ((rc = upload_desc(e, m, s))) return rc;
  }
  long long live_nodes = 0;
  std::vector<int> ids, evals, prep_ids;
  std::vector<ExpmJob> jobs;
  std::vector<int> readers;
  for (;;) {
    long long iter_nodes = 0;
    bool any_read = false, any_prep = false;
    live_nodes = 0;
    ids.clear();
    for (int m = 0; m < e.count; ++m) {
      const Member& M = e.mem[m];
      if (M.wait == W_DONE) continue;
      live_nodes += M.c->nodes;
      if (M.wait == W_ITER) {
        iter_nodes += M.c->nodes;
        ids.push_back(m);
      } else if (M.wait == W_READ) {
        any_read = true;
      } else if (M.wait == W_PREP) {
        any_prep = true;
      }
    }
    if (ids.empty() && !any_read && !any_prep) break;
    const bool drain = (any_read || any_prep) && (ids.empty() || (double)iter_nodes < e.theta * (double)live_nodes);
    if (!drain) {
      if ((rc = launch_iteration(e, ids, s))) return rc;
      for (int m : ids) {
        Member& M = e.mem[m];
        if (++M.j_dev >= M.m_cur) {
          M.cst = CS_PREP;
          M.wait = W_PREP;
        }
      }
      continue;
    }
    // serve every member that waits on the host, until all iterate or are done
    for (;;) {
      bool pending = false;
      for (const Member& M : e.mem) pending = pending || M.wait == W_READ || M.wait == W_PREP;
      if (!pending) break;
      if ((rc = launch_prep_batch(e, jobs, prep_ids, s))) return rc;
      if ((rc = gather(e, s))) return rc;
      readers.clear();
      for (int m = 0; m < e.count; ++m)
        if (e.mem[m].wait == W_READ) readers.push_back(m);
      evals.clear();
      for (int m : readers) {
        e.mem[m].wait = W_NONE;
        if ((rc = on_read(e, m, e.h_gather + (long long)m * ENS_GATHER, o, evals, s))) return rc;
      }
      if ((rc = launch_eval_batch(e, evals, s))) return rc;
    }
  }
  if ((rc = join_all(e, s))) return rc;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SW_ECUDA;
  e.ring_off = 0;
  drain_events(e);
  e.st.launches += member_launches(e) - l0;
  if (stats)
    for (int m = 0; m < e.count; ++m) stats[m] = e.mem[m].acc;
  return cuda_rc(cudaGetLastError());
}

// ---------------------------------------------------------------- autotuner
namespace {

// time `iters` batched iterations of the members in ids from basis index 0 (ms per iteration)
int time_iterations(Ens& e, const std::vector<int>& ids, int iters, cudaStream_t s, double* ms) {
  int rc;
  for (int m : ids)
    if ((rc = upload_j(e, m, 0, s))) return rc;
  if ((rc = launch_iteration(e, ids, s))) return rc;   // warm-up
  for (int m : ids)
    if ((rc = upload_j(e, m, 0, s))) return rc;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return SW_ECUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return SW_ECUDA;
  }
  cudaEventRecord(a, s);
  for (int it = 0; it < iters && rc == SW_OK; ++it) rc = launch_iteration(e, ids, s);
  cudaEventRecord(b, s);
  float t = 0.f;
  if (rc == SW_OK && cudaEventSynchronize(b) != cudaSuccess) rc = SW_ECUDA;
  if (rc == SW_OK) cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  e.ring_off = 0;
  if (rc == SW_OK) {
    // a wait that gave up would make the timing meaningless
    EnsCtl ctl{};
    if (cudaMemcpy(&ctl, e.d_ctl, sizeof(EnsCtl), cudaMemcpyDeviceToHost) != cudaSuccess) return SW_ECUDA;
    if (ctl.error) return SW_ETIMEOUT;
  }
  *ms = t / std::max(1, iters);
  return rc;
}

}  // namespace

int ens_tune(Ens& e, double* const* q, int iters, cudaStream_t s, int* chosen_block) {
  int rc;
  const bool prof = e.prof;
  e.prof = false;
  struct Restore {
    Ens& e;
    bool p;
    ~Restore() { e.prof = p; }
  } restore{e, prof};
  iters = std::max(1, std::min(iters, 32));
  // a unit start vector per member, lin tables at its state, a plain operator (p = 1, no b)
  for (int m = 0; m < e.count; ++m) {
    Ctx& c = *e.mem[m].c;
    if ((rc = ensure_krylov(c, 64))) return rc;
    if ((rc = launch_linearize(c, q[m], s))) return rc;
    if ((rc = launch_norm2(c, q[m], c.n, c.d_scal + S_BETA, 0.0, nullptr, 0, nullptr, s))) return rc;
    if ((rc = launch_scale_inv(c, c.d_V, q[m], c.d_scal + S_BETA, c.n, nullptr, s))) return rc;
    double zero[MAX_NB] = {};
    if ((rc = launch_set_tail(c, c.d_V, c.n, 1, zero, s))) return rc;
    if (cudaMemsetAsync(c.d_flags, 0, sizeof(int) * 2, s) != cudaSuccess) return SW_ECUDA;
    EnsDesc& d = e.hdesc[m];
    d.V = c.d_V;
    d.ldv = c.ldv;
    d.H = c.d_H;
    d.ldh = c.ldh;
    d.cdot = c.d_cdot;
    d.vpart = c.d_vpart;
    d.flags = c.d_flags;
    d.lf = c.d_lin_face;
    d.ln = c.d_lin_node;
    d.tol = 0.0;
    d.scale = 1.0;
    d.nu = 0.0;
    d.p = 1;
    for (int l = 0; l < MAX_NB; ++l) d.b[l] = nullptr;
  }
  // classes: members with the same (n_e, p), largest work first
  std::map<std::pair<int, int>, std::vector<int>> cls;
  for (int m = 0; m < e.count; ++m) cls[{e.mem[m].c->ne, e.mem[m].c->ns}].push_back(m);
  std::vector<std::vector<int>> order;
  for (auto& kv : cls) order.push_back(kv.second);
  std::sort(order.begin(), order.end(), [&](const std::vector<int>& a, const std::vector<int>& b) {
    return e.mem[a[0]].c->nodes * (long long)a.size() > e.mem[b[0]].c->nodes * (long long)b.size();
  });
  std::vector<int> all(e.count);
  for (int m = 0; m < e.count; ++m) all[m] = m;
  double best_all = 1e300;
  int best_block = e.block;
  std::vector<sw_ens_tiles> best_tiles(e.count);
  for (int block : kBlocks) {
    if ((rc = ensure_graph(e, block))) return rc;
    e.block = block;
    for (int m = 0; m < e.count; ++m) e.mem[m].tiles = default_tiles(block);
    for (int m = 0; m < e.count; ++m)
      if ((rc = upload_desc(e, m, s))) return rc;
    for (const std::vector<int>& members : order) {
      const int opts_face[4] = {block, 2 * block, 4 * block, 8 * block};
      const int opts_vol[3] = {1, 2, 4};
      const int opts_vec[3] = {4 * block, 16 * block, 64 * block};
      sw_ens_tiles cur = e.mem[members[0]].tiles;
      double cur_ms = 0.0;
      for (int m : members)
        if ((rc = upload_desc(e, m, s))) return rc;
      if ((rc = time_iterations(e, members, iters, s, &cur_ms))) return rc;
      for (int param = 0; param < 3; ++param) {
        const int nopt = (param == 0) ? 4 : 3;
        for (int k = 0; k < nopt; ++k) {
          sw_ens_tiles t = cur;
          if (param == 0) t.face_pts = opts_face[k];
          else if (param == 1) t.vol_tiles = opts_vol[k];
          else t.vec_len = opts_vec[k];
          if (t.face_pts == cur.face_pts && t.vol_tiles == cur.vol_tiles && t.vec_len == cur.vec_len) continue;
          for (int m : members) {
            e.mem[m].tiles = t;
            if ((rc = upload_desc(e, m, s))) return rc;
          }
          double ms = 0.0;
          if ((rc = time_iterations(e, members, iters, s, &ms))) return rc;
          if (ms < cur_ms) {
            cur_ms = ms;
            cur = t;
          }
        }
      }
      for (int m : members) {
        e.mem[m].tiles = cur;
        if ((rc = upload_desc(e, m, s))) return rc;
      }
    }
    double ms_all = 0.0;
    if ((rc = time_iterations(e, all, iters, s, &ms_all))) return rc;
    if (ms_all < best_all) {
      best_all = ms_all;
      best_block = block;
      for (int m = 0; m < e.count; ++m) best_tiles[m] = e.mem[m].tiles;
    }
  }
  e.block = best_block;
  for (int m = 0; m < e.count; ++m) {
    e.mem[m].tiles = best_tiles[m];
    if ((rc = upload_desc(e, m, s))) return rc;
    if ((rc = upload_j(e, m, 0, s))) return rc;
    e.mem[m].j_dev = -1;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return SW_ECUDA;
  e.ring_off = 0;
  if (chosen_block) *chosen_block = best_block;
  return SW_OK;
}

}  // namespace swepi

// ====================================================================== C ABI
using namespace swepi;

namespace {
cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// zero every member's phase counters and tickets (no launch in flight)
int reset_dyn(sw_ens* e) {
  if (cudaDeviceSynchronize() != cudaSuccess) return SW_ECUDA;
  if (cudaMemset(e->d_dyn, 0, sizeof(EnsDyn) * e->count) != cudaSuccess) return SW_ECUDA;
  e->hdyn.assign(e->count, EnsDyn{});
  e->dyn_stale = false;
  return SW_OK;
}

void ens_release(sw_ens* e) {
  for (int i = 0; i < 3; ++i) {
    if (e->gexec[i]) cudaGraphExecDestroy(e->gexec[i]);
    if (e->graph[i]) cudaGraphDestroy(e->graph[i]);
  }
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  cudaFree(e->d_desc);
  cudaFree(e->d_dyn);
  cudaFree(e->d_list);
  cudaFree(e->d_ctl);
  cudaFree(e->d_gsrc);
  cudaFree(e->d_gather);
  cudaFree(e->d_jobs);
  cudaFree(e->d_upart);
  for (cudaEvent_t ev : e->ev_pool) cudaEventDestroy(ev);
  for (cudaEvent_t ev : e->mevent)
    if (ev) cudaEventDestroy(ev);
  if (e->start_event) cudaEventDestroy(e->start_event);
  for (cudaStream_t st : e->mstream)
    if (st) cudaStreamDestroy(st);
  if (e->h_gather) cudaFreeHost(e->h_gather);
  if (e->h_ring) cudaFreeHost(e->h_ring);
  delete e;
}
}  // namespace

extern "C" {

int sw_ens_create(int members, const sw_ctx_t* ctxs, sw_ens_t* out) {
  if (!out || !ctxs || members < 1 || members > ENS_MAX) return SW_EINVAL;
  *out = nullptr;
  for (int m = 0; m < members; ++m) {
    if (!ctxs[m] || ctxs[m]->ns < 4 || ctxs[m]->ns > 6) return SW_EINVAL;
    for (int k = 0; k < m; ++k)
      if (ctxs[k] == ctxs[m]) return SW_EINVAL;
  }
  sw_ens* e = new (std::nothrow) sw_ens();
  if (!e) return SW_ENOMEM;
  e->count = members;
  e->mem.resize(members);
  e->hdesc.assign(members, EnsDesc{});
  e->hdyn.assign(members, EnsDyn{});
  if (cudaGetDevice(&e->device) != cudaSuccess) {
    ens_release(e);
    return SW_ECUDA;
  }
  long long max_upart = 0;
  std::vector<GatherSrc> gsrc(members);
  for (int m = 0; m < members; ++m) {
    Ctx& c = *ctxs[m];
    Member& M = e->mem[m];
    M.c = &c;
    M.tiles = default_tiles(e->block);
    EnsDesc& d = e->hdesc[m];
    d.ns = c.ns;
    d.nodes = c.nodes;
    d.nelem = c.nelem;
    d.nfacepts = c.nfacepts;
    d.n = c.n;
    d.lines = c.d_lines;
    d.fc = c.d_face_coef;
    d.fb = c.d_fb;
    d.dc = c.dc;
    d.p = 1;
    max_upart = std::max(max_upart, (c.n + MAX_NB + 127) / 128 + 1);
    gsrc[m] = GatherSrc{nullptr, nullptr};
  }
  // every member needs its Krylov scalars and flags before the gather table is built
  for (int m = 0; m < members; ++m) {
    int rc = ensure_krylov(*ctxs[m], 16);
    if (rc) {
      ens_release(e);
      return rc;
    }
    gsrc[m] = GatherSrc{ctxs[m]->d_scal, ctxs[m]->d_flags};
  }
  e->upart_stride = max_upart;
  e->ring_cap = size_t(8) << 20;
  bool ok = cudaMalloc(&e->d_desc, sizeof(EnsDesc) * members) == cudaSuccess &&
            cudaMalloc(&e->d_dyn, sizeof(EnsDyn) * members) == cudaSuccess &&
            cudaMalloc(&e->d_list, sizeof(EnsList)) == cudaSuccess &&
            cudaMalloc(&e->d_ctl, sizeof(EnsCtl)) == cudaSuccess &&
            cudaMalloc(&e->d_gsrc, sizeof(GatherSrc) * members) == cudaSuccess &&
            cudaMalloc(&e->d_gather, sizeof(double) * (members * ENS_GATHER + 2)) == cudaSuccess &&
            cudaMalloc(&e->d_jobs, sizeof(ExpmJob) * members) == cudaSuccess &&
            cudaMalloc(&e->d_upart, sizeof(double) * max_upart * members) == cudaSuccess &&
            cudaMallocHost(&e->h_gather, sizeof(double) * (members * ENS_GATHER + 2)) == cudaSuccess &&
            cudaMallocHost(&e->h_ring, e->ring_cap) == cudaSuccess;
  if (!ok) {
    ens_release(e);
    return SW_ENOMEM;
  }
  for (int m = 0; m < members; ++m) e->hdesc[m].upart = e->d_upart + (long long)m * max_upart;
  ok = cudaMemset(e->d_dyn, 0, sizeof(EnsDyn) * members) == cudaSuccess &&
       cudaMemset(e->d_ctl, 0, sizeof(EnsCtl)) == cudaSuccess &&
       cudaMemset(e->d_list, 0, sizeof(EnsList)) == cudaSuccess &&
       cudaMemcpy(e->d_gsrc, gsrc.data(), sizeof(GatherSrc) * members, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  e->mstream.assign(members, nullptr);
  e->mevent.assign(members, nullptr);
  e->dirty.assign(members, 0);
  ok = ok && cudaEventCreateWithFlags(&e->start_event, cudaEventDisableTiming) == cudaSuccess;
  for (int m = 0; m < members && ok; ++m)
    ok = cudaStreamCreateWithFlags(&e->mstream[m], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e->mevent[m], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    ens_release(e);
    return SW_ECUDA;
  }
  *out = e;
  return SW_OK;
}

int sw_ens_free(sw_ens_t e) {
  if (!e) return SW_EINVAL;
  cudaDeviceSynchronize();
  ens_release(e);
  return SW_OK;
}

int sw_ens_set_block(sw_ens_t e, int block) {
  if (!e || block_index(block) < 0) return SW_EINVAL;
  e->block = block;
  return SW_OK;
}

int sw_ens_set_tiles(sw_ens_t e, int member, const sw_ens_tiles* t) {
  if (!e || !t || member < 0 || member >= e->count || !tiles_valid(*t)) return SW_EINVAL;
  e->mem[member].tiles = *t;
  return SW_OK;
}

int sw_ens_get_tiles(sw_ens_t e, int member, sw_ens_tiles* t) {
  if (!e || !t || member < 0 || member >= e->count) return SW_EINVAL;
  *t = e->mem[member].tiles;
  return SW_OK;
}

int sw_ens_set_policy(sw_ens_t e, double theta) {
  if (!e || !(theta >= 0.0) || !(theta <= 1.0)) return SW_EINVAL;
  e->theta = theta;
  return SW_OK;
}

int sw_ens_tune(sw_ens_t e, double* const* q_dev, int iters, int* block, void* stream) {
  if (!e || !q_dev) return SW_EINVAL;
  for (int m = 0; m < e->count; ++m)
    if (!q_dev[m]) return SW_EINVAL;
  int rc = e->dyn_stale ? reset_dyn(e) : SW_OK;
  if (rc) return rc;
  rc = ens_tune(*e, q_dev, iters, as_stream(stream), block);
  if (rc) e->dyn_stale = true;
  return rc;
}

int sw_ens_epi_run(sw_ens_t e, int steps, const int* orders, const double* dts, double* const* q_dev,
                   const sw_kiops_opts* opts, sw_kiops_stats* stats, void* stream) {
  if (!e || !orders || !dts || !q_dev || steps < 0) return SW_EINVAL;
  sw_kiops_opts o = opts ? *opts : default_opts();
  if (o.iop != 2 || o.m_min < 1 || o.m_max < o.m_min || o.m_max > 150 || !(o.tol > 0)) return SW_EINVAL;
  for (int m = 0; m < e->count; ++m) {
    const Ctx& c = *e->mem[m].c;
    if (!q_dev[m] || orders[m] < 2 || orders[m] > 6 || !std::isfinite(dts[m]) || !(dts[m] > 0)) return SW_EINVAL;
    // members run the FP64 split JVP with the plain adaptive rule
    if (c.jvp_mode != 1 || c.controller) return SW_EINVAL;
  }
  TraceRange trace("ensemble EPI run");
  int rc = e->dyn_stale ? reset_dyn(e) : SW_OK;
  if (rc) return rc;
  rc = ens_run(*e, steps, orders, dts, q_dev, o, stats, as_stream(stream));
  if (rc) e->dyn_stale = true;
  return rc;
}

int sw_ens_set_wait_test(sw_ens_t e, double limit_s, int extra) {
  if (!e || !(limit_s >= 0.0) || limit_s > 2.0 || extra < 0 || extra > 1) return SW_EINVAL;
  // no launch of this ensemble is in flight between calls; writing the control
  // block also clears an earlier give-up
  if (cudaDeviceSynchronize() != cudaSuccess) return SW_ECUDA;
  EnsCtl ctl{};
  ctl.extra = (unsigned int)extra;
  ctl.limit_ns = (unsigned long long)(limit_s * 1e9);
  if (cudaMemcpy(e->d_ctl, &ctl, sizeof(EnsCtl), cudaMemcpyHostToDevice) != cudaSuccess) return SW_ECUDA;
  return reset_dyn(e);
}

int sw_ens_profile(sw_ens_t e, int enable) {
  if (!e) return SW_EINVAL;
  e->prof = enable != 0;
  return SW_OK;
}

int sw_ens_stats_read(sw_ens_t e, sw_ens_stats* out) {
  if (!e || !out) return SW_EINVAL;
  *out = e->st;
  out->block = e->block;
  const int bi = block_index(e->block);
  out->ctas = (bi >= 0) ? e->ctas[bi] : 0;
  return SW_OK;
}

}  // extern "C"

namespace swepi {
// this translation unit's check word (bounds-checked builds; sw_check_status)
SW_CHECK_READER(check_word_ensemble)
}  // namespace swepi
