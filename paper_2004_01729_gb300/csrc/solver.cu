// Host side of libftcc: contexts, batches of problem instances, the
// contraction engine, the S-kernel schedule, the fixed-point iteration and
// the C ABI of include/ftcc.h.
//
// A batch holds nz instances (one per context) that share the orbital
// counts, the tau grid and the arithmetic; every per-instance tensor carries
// an instance index z in front, so one launch of each contraction serves the
// whole batch and one CUDA graph replays an iteration of all instances.
#include <algorithm>
#include <system_error>
#include <atomic>
#include <thread>
#include <array>
#include <tuple>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <unordered_map>
#include <memory>
#include <string>
#include <vector>

#include "ftcc_internal.h"

namespace ftcc {

void* Alloc::get(size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (custom) return a.alloc(bytes, a.user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}
void Alloc::put(void* p) {
  if (!p) return;
  if (custom) a.release(p, a.user);
  else cudaFree(p);
}

// Status carried through the host code: the first failure wins.
struct Fail {
  ftcc_status s;
  std::string msg;
};

inline bool is_hole(char c) { return c >= 'i' && c <= 'n'; }

template <class T> struct Solver;
struct Batch;
struct SpTables;

}  // namespace ftcc

struct ftcc_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  ftcc::Alloc alloc;
  std::string err;
  int* dev_err = nullptr;
  // system
  int N = 0;
  ftcc::Buf h, eri, eps;
  // prepared problem: the batch this context belongs to and its index in it
  std::shared_ptr<ftcc::Batch> batch;
  int member = 0;
  // tensor-core GEMM autotuner: (kind, batch, M, N, K, transposed output,
  // accumulate) -> (tile width, K split), kept for the context's lifetime so
  // that repeated solves in one context take the same launches (and round
  // the same way)
  std::map<std::array<int, 7>, std::pair<int, int>> tuned;
  // conserved charge of every spin orbital (up to four integer components,
  // component k taken modulo charge_mod[k] when that is > 0), for systems
  // whose orbitals all carry distinct charges (UEG: momentum and S_z; k-space
  // Hubbard ring: crystal momentum mod L and S_z); empty otherwise
  std::vector<std::array<int, 4>> charge;
  int charge_mod[4] = {0, 0, 0, 0};
  // block-sparse tables of these charges (implied-index table, lists of valid
  // positions, pair sectors), built by the first block-sparse prepare and
  // kept until the system is rebuilt
  std::shared_ptr<ftcc::SpTables> sptab;
  // pinned host copy of the per-instance convergence state of the batch
  // this context is home to (written by each iteration's graph tail)
  double* pin_state = nullptr;
  size_t pin_state_n = 0;
  // a second stream for work that may overlap the main stream's (created on
  // first use; joined back through ev_join before the main stream goes on)
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  ftcc::Buf get(size_t bytes) {
    ftcc::Buf b;
    b.p = alloc.get(bytes);
    b.bytes = b.p ? bytes : 0;
    return b;
  }
  void put(ftcc::Buf& b) {
    if (b.p) alloc.put(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
};

namespace ftcc {

static ftcc_status fail(ftcc_ctx* c, ftcc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CU(...)                                                                                    \
  do {                                                                                             \
    cudaError_t e_ = (__VA_ARGS__);                                                                \
    if (e_ != cudaSuccess) throw Fail{FTCC_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

static void ensure(ftcc_ctx* c, Buf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return;
  if (b.p) {
    CU(cudaStreamSynchronize(c->st));
    c->put(b);
  }
  b = c->get(bytes);
  if (!b.p) throw Fail{FTCC_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
}

// A tensor view for the engine: pointer + index letters (row-major in that
// order); `fixed` marks operands that do not change between iterations
// (integral and Fock blocks), whose packed GEMM forms are cached.
template <class T>
struct Tn {
  T* p;
  const char* L;
  bool fixed = false;
};

struct PackKey {
  const void* p;
  std::string rows, cols;
  long long ld;
  int kind;
  bool operator<(const PackKey& o) const {
    if (p != o.p) return p < o.p;
    if (rows != o.rows) return rows < o.rows;
    if (cols != o.cols) return cols < o.cols;
    if (ld != o.ld) return ld < o.ld;
    return kind < o.kind;
  }
};

// One prepared problem instance: reference quantities of (system, beta, mu).
struct Inst {
  ftcc_ctx* ctx = nullptr;       // owner of the Hamiltonian
  double beta = 0, mu = 0, hstep = 0, omega0 = 0, omega1 = 0;
  std::vector<double> n_host, nbar_host;
  Buf n, nbar, f, fbar, facO, facV;
  int conv_iter = -1;
};

// Charge sectors of ordered orbital pairs (p, q), grouped by q_p + q_q
// (sum) or q_p - q_q (difference), with the summed-index list of each sector
// and the tiles of its products (see sector_gemm_kernel).
struct SecTab {
  Buf ent, kl, sec, work, work_small;
  int nwork = 0, nwork_small = 0;   // work_small: one item per sector of at most 16 pairs
  double flops = 0;   // 2 sum_s rows_s^2 K_s per slice
};

// Block-sparse tables of one set of orbital charges (option block_sparse): the
// implied-index table imp[a][b][c] (int16, N^3), lists of valid positions and
// the pair-charge sectors.  SpTables owns the device buffers (cached on the
// context); a batch holds a copy of the view and a reference to the owner.
struct SpTableView {
  Buf imp;
  Buf canon;                     // canonical doubles positions (i < j, a < b) of the N^3 storage
  long long ncanon = 0;
  Buf vl1, voff1, vl2, voff2;    // per orbital p: valid (m, q) of (m, q, p) and of (p, m, q)
  // positions (p0, p1, p2) of the N^3 storage whose (p0, p1, p2), (p0, p2, p1)
  // or (p1, p2, p0) has an implied index (the element-wise kernels' lists)
  Buf vall, vswap, vrot;
  int nvall = 0, nvswap = 0, nvrot = 0;
  SecTab ssum, sdiff, ssum_u;   // ssum_u: unordered pairs p < q only
};

struct SpTables : SpTableView {
  ftcc_ctx* home = nullptr;
  int n = 0;
  ~SpTables();
};

struct Batch : SpTableView {
  ftcc_ctx* home = nullptr;      // allocator, stream and error flag of the batch
  std::vector<Inst> inst;
  int nz = 0, N = 0, no = 0, nv = 0, ng = 0, prec = 0;
  ftcc_options opt{};
  std::vector<int> O, V;
  Buf idxO, idxV, em, ep, hz, V64, F64, state, live;
  std::vector<int> live_host;     // 0 once an instance diverged (frozen, reported DIVERGED)
  std::unique_ptr<Solver<float>> s32;
  std::unique_ptr<Solver<double>> s64;
  int active = 0;                // 0 = FP64 solver, 1 = FP32 solver
  // adjoint state (FP64): weighted multipliers m = g lambda / beta, their
  // back-propagated cotangents u, and the S-kernel VJP
  Buf m1, m2, mn1, mn2, u1, u2, tb1, tb2, dE1, cz, lpart;
  Buf facOz, facVz, epsz;        // stacked [nz][no], [nz][nv], [nz][N] for the response
  bool lambda_done = false;
  // the response of every member, computed once per converged multipliers
  bool resp_done = false;
  std::vector<ftcc_adjoint_result> resp;
  std::vector<std::vector<double>> resp_rdm;
  bool adjoint_fp32 = false;     // the multipliers live on the FP32 solver (mixed adjoint)
  int lambda_iterations = 0;
  double prof_ms[8] = {0}, prof_bytes[8] = {0}, prof_flops[8] = {0};
  long long prof_launches[8] = {0};
  int iterations = 0, refine_iterations = 0, polish_iterations = 0;
  bool polishing = false;        // the FP32 solver runs the BF16X3 polishing phase
  double ms_total = 0;
  int ms_count = 0;
  bool solved = false;
  bool solved_live = false;   // every live member converged (diverged members are frozen)
  int quad = FTCC_QUAD_SIMPSON;   // integral form (Simpson fixed point) or an RK march of Eq. smud
  // block-sparse storage (option block_sparse)
  bool sparse = false;
  std::shared_ptr<SpTables> sp_owner;
  ~Batch();
};

constexpr int kStateStride = 8 + 256;

// kernel classes of the per-iteration timing
enum { kClsScatter = 0, kClsPack, kClsGemmTc, kClsGemmSimt, kClsPropagate, kClsOther, kClsSector, kNumCls };
const char* const kClsName[kNumCls] = {"layout:scatter", "layout:pack", "gemm_tc_kernel",
                                       "gemm_simt_kernel", "propagate_kernel", "other", "sector_gemm_kernel"};

template <class T>
struct Solver {
  Batch* b;
  ftcc_ctx* h_;
  int gk;                  // GEMM_F64 for double; GEMM_TF32 / GEMM_BF16X3 for float
  int nz = 1, no = 0, nv = 0, ng = 0, nxc = 0;   // nxc = tau points per S pass
  bool sp = false;         // block-sparse storage (FP64 only): singles [N], doubles [N^3] per tau point
  long long n1() const { return sp ? no : static_cast<long long>(no) * nv; }
  long long n2() const { return sp ? static_cast<long long>(no) * no * no : static_cast<long long>(no) * no * nv * nv; }
  bool stream = false;                            // S kept per tau chunk, propagation chained
  Buf ch1, ch2;                                   // chain state [5][size] of the singles / doubles
  int nx = 0;              // tau points of the current pass
  std::map<std::string, Buf> Vb, Fb;
  Buf t1, t2, S1, S2;
  Buf tt, ta, X, Wmnij, Wabef, Wmbej, Fae, Fmi, Fme, Ft, Ft2, Y, R, R2;
  // the ladders over unordered pairs: tau, W_mnij, W_abef and their result
  // packed [zx][pair][pair], <mn||ef> packed once, and the pair tables
  Buf tp, WAmn, WAef, Lp, Vp, pairsO, pairsV;
  Buf pA, pB, pA2, pB2, Ct, skw;
  std::map<PackKey, std::pair<Buf, Buf>> packed;   // cached packs of fixed operands
  Buf part1, part2;
  int nb1 = 0, nb2 = 0;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;   // the captured iteration gexec was made from (a batched step embeds it)
  unsigned graph_gen = 0;        // bumped at every capture
  bool warm = false;       // one uncaptured iteration has sized every workspace
  int graph_nodes = 0;     // kernels in one captured iteration
  long long gemm_flops = 0;   // algorithmic GEMM flops counted while `counting`
  bool counting = false;

  // Tape of one S-kernel pass, replayed backwards for the vector-Jacobian
  // product (the lambda equations are the transpose of the S kernel).
  struct Op {
    int kind;                  // 0 contract, 1 scatter, 2 tau build, 3 X build
    T* C;
    std::string Lc;
    const T* A;
    std::string La;
    const T* B;
    std::string Lb;
    T* C2;
    double alpha, beta;
    std::string anti;
  };
  std::vector<Op> tape;
  bool recording = false;

  // Kernel timing: CUDA events around every launch of the iteration (inside
  // the captured graph as event nodes), summed per kernel class with the
  // algorithmic bytes and flops of each launch.
  struct ProfRec {
    int cls;
    cudaEvent_t e0, e1;
    double bytes, flops;
  };
  bool profiling = false;
  std::vector<ProfRec> prof;
  size_t prof_next = 0;
  template <class F>
  void timed_launch(int cls, double bytes, double flops, F&& launch) {
    if (!profiling) {
      launch();
      return;
    }
    if (prof_next == prof.size()) {
      ProfRec r{};
      CU(cudaEventCreate(&r.e0));
      CU(cudaEventCreate(&r.e1));
      prof.push_back(r);
    }
    ProfRec& r = prof[prof_next++];
    r.cls = cls;
    r.bytes = bytes;
    r.flops = flops;
    // inside a stream capture the records must become graph nodes of their own
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(st(), &cs));
    const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    CU(cudaEventRecordWithFlags(r.e0, st(), flags));
    launch();
    CU(cudaEventRecordWithFlags(r.e1, st(), flags));
  }
  std::map<const void*, T*> bar;            // forward buffer -> its adjoint
  std::map<const void*, Buf> fixed_bar;     // integral / Fock block -> adjoint (when wanted)
  bool want_fixed_bar = false;
  // block-sparse transpose: the forward intermediates of the amplitudes at
  // vjp_fwd_key (nx = vjp_fwd_nx slices) are still in their buffers.  Only
  // the lambda sweep and the response set vjp_fwd_reuse (the amplitudes are
  // fixed there); every forward S evaluation clears the key.
  bool vjp_fwd_reuse = false;
  const void* vjp_fwd_key = nullptr;
  int vjp_fwd_nx = 0;
  Buf btt, bta, bX, bWmnij, bWabef, bWmbej, bY, bFae, bFmi, bFme, bFt, bFt2, bR, bR2, bD, bP, bQ, ones, sx1, sx2;

  Solver(Batch* batch, int kind) : b(batch), h_(batch->home), gk(kind) {}

  // Change the tensor-core arithmetic of the contractions (TF32 -> BF16X3
  // for the polishing phase) keeping the amplitudes: the operand packs of the
  // old kind are released and the next iteration runs uncaptured (sizing the
  // new kind's workspaces) before a new graph is captured.
  void set_kind(int kind) {
    if (kind == gk) return;
    gk = kind;
    for (auto& kv : packed) {
      h_->put(kv.second.first);
      h_->put(kv.second.second);
    }
    packed.clear();
    for (auto& e : amp_cache) {
      h_->put(e.a);
      h_->put(e.b);
    }
    amp_cache.clear();
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    if (graph) cudaGraphDestroy(graph);
    graph = nullptr;
    warm = false;
    graph_nodes = 0;
  }
  ~Solver() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& kv : Vb) h_->put(kv.second);
    for (auto& kv : Fb) h_->put(kv.second);
    for (auto& kv : packed) {
      h_->put(kv.second.first);
      h_->put(kv.second.second);
    }
    Buf* bs[] = {&t1, &t2, &S1, &S2, &ch1, &ch2, &tt, &ta, &X, &Wmnij, &Wabef, &Wmbej, &Fae, &Fmi, &Fme, &Ft, &Ft2, &Y,
                 &R, &R2, &bR, &bR2, &tuneC, &tp, &WAmn, &WAef, &Lp, &Vp, &pairsO, &pairsV,
                 &pA, &pB, &pA2, &pB2, &Ct, &skw, &part1, &part2, &btt, &bta, &bX, &bWmnij, &bWabef, &bWmbej,
                 &bY, &bFae, &bFmi, &bFme, &bFt, &bFt2, &bD, &bP, &bQ, &ones, &sx1, &sx2};
    for (Buf* q : bs) h_->put(*q);
    for (auto& e : amp_cache) {
      h_->put(e.a);
      h_->put(e.b);
    }
    for (auto& kv : fixed_bar) h_->put(kv.second);
    for (auto& kv : perm_cache) h_->put(kv.second);
    for (auto& r : prof) {
      cudaEventDestroy(r.e0);
      cudaEventDestroy(r.e1);
    }
  }
  cudaStream_t st() const { return h_->st; }
  // fork: the side stream waits for everything enqueued on st() so far
  cudaStream_t side_begin() {
    if (!h_->st2) {
      CU(cudaStreamCreateWithFlags(&h_->st2, cudaStreamNonBlocking));
      CU(cudaEventCreateWithFlags(&h_->ev_fork, cudaEventDisableTiming));
      CU(cudaEventCreateWithFlags(&h_->ev_join, cudaEventDisableTiming));
    }
    CU(cudaEventRecord(h_->ev_fork, st()));
    CU(cudaStreamWaitEvent(h_->st2, h_->ev_fork, 0));
    return h_->st2;
  }
  // join: st() waits for the side stream's work
  void side_end() {
    CU(cudaEventRecord(h_->ev_join, h_->st2));
    CU(cudaStreamWaitEvent(st(), h_->ev_join, 0));
  }

  long long dimof(char ch) const {
    if (ch == 'z') return nz;
    if (ch == 'x') return nx;
    // unordered pairs (p < q) of hole-like (I, J) and particle-like (A, E) letters
    if (ch == 'I' || ch == 'J') return static_cast<long long>(no) * (no - 1) / 2;
    if (ch == 'A' || ch == 'E') return static_cast<long long>(nv) * (nv - 1) / 2;
    if (is_hole(ch)) return no;
    return nv;
  }
  std::vector<long long> strides_of(const char* L) const {
    const int n = static_cast<int>(strlen(L));
    std::vector<long long> s(n);
    long long acc = 1;
    for (int k = n - 1; k >= 0; --k) {
      s[k] = acc;
      acc *= dimof(L[k]);
    }
    return s;
  }
  static std::string classes(const char* L) {
    std::string s;
    for (const char* q = L; *q; ++q)
      if (*q != 'z') s += is_hole(*q) ? 'o' : 'v';
    return s;
  }
  T* V(const char* L) {
    auto it = Vb.find(classes(L));
    if (it == Vb.end()) throw Fail{FTCC_ERR_STATE, "integral block " + classes(L) + " not built"};
    return static_cast<T*>(it->second.p);
  }
  T* F(const char* L) {
    auto it = Fb.find(classes(L));
    if (it == Fb.end()) throw Fail{FTCC_ERR_STATE, "fock block " + classes(L) + " not built"};
    return static_cast<T*>(it->second.p);
  }

  // dst (letters Ld) = beta * dst + alpha * P(src with letters Ls); letters of
  // dst missing from src are broadcast.  anti names letter pairs of dst to
  // antisymmetrise: "", "ij", "ab" or "ijab".
  // Fixed (integral or Fock) blocks stored again in another letter order for
  // the broadcast copies of the S kernel (at most kPermCacheBytes in all).
  static constexpr size_t kPermCacheBytes = size_t(4) << 30;
  std::map<std::pair<const void*, std::string>, Buf> perm_cache;
  size_t perm_cache_bytes = 0;

  // dst = beta dst + alpha src when dst's trailing letters form one block
  // that src holds contiguously in the same order (its other letters leading
  // in dst, the ones src lacks broadcast): one vectorised copy per leading
  // index.  False when the layouts do not have that form.
  bool block_copy(T* dst, const char* Ld, const T* src, const char* Ls, double alpha, double beta) {
    const int nd = static_cast<int>(strlen(Ld)), ns = static_cast<int>(strlen(Ls));
    int k = 0;
    while (k < nd && k < ns && Ld[nd - 1 - k] == Ls[ns - 1 - k]) ++k;
    if (k == 0 || nd - k > kMaxL) return false;
    long long B = 1;
    for (int q = nd - k; q < nd; ++q) B *= dimof(Ld[q]);
    BlockCopyDesc bd{};
    bd.nouter = nd - k;
    const auto ss = strides_of(Ls);
    int found = 0;
    long long nout = 1;
    for (int q = 0; q < bd.nouter; ++q) {
      bd.dim[q] = dimof(Ld[q]);
      nout *= bd.dim[q];
      const char* f = strchr(Ls, Ld[q]);
      if (f) {
        if (f - Ls >= ns - k) return false;
        bd.sst[q] = ss[f - Ls];
        ++found;
      } else {
        bd.sst[q] = 0;
      }
    }
    if (found != ns - k || nout > 65535 || B < 1024) return false;
    const double reads = 1.0 + (beta != 0.0 ? 1.0 : 0.0);
    timed_launch(kClsScatter, static_cast<double>(nout) * B * (reads + 1) * sizeof(T), 0.0,
                 [&] { CU(launch_block_copy<T>(dst, src, B, bd, alpha, beta, st())); });
    return true;
  }

  void scatter(T* dst, const char* Ld, const T* src, const char* Ls, double alpha, double beta, const char* anti) {
    if (recording) tape.push_back(Op{1, dst, Ld, src, Ls, nullptr, "", nullptr, alpha, beta, anti});
    if (!*anti) {
      if (block_copy(dst, Ld, src, Ls, alpha, beta)) return;
      // a fixed block broadcast in another order: copy it once into dst's
      // order (without the broadcast letters), then block copies
      if (is_fixed(src)) {
        std::string Lt;
        for (const char* q = Ld; *q; ++q)
          if (strchr(Ls, *q)) Lt += *q;
        if (Lt.size() == strlen(Ls)) {
          const auto key = std::make_pair(static_cast<const void*>(src), Lt);
          auto it = perm_cache.find(key);
          long long n = 1;
          for (const char* q = Ls; *q; ++q) n *= dimof(*q);
          const size_t bytes = static_cast<size_t>(n) * sizeof(T);
          if (it == perm_cache.end() && perm_cache_bytes + bytes <= kPermCacheBytes) {
            Buf b;
            ensure(h_, b, bytes);
            scatter_permute(static_cast<T*>(b.p), Lt.c_str(), src, Ls, 1.0, 0.0, "");
            perm_cache_bytes += bytes;
            it = perm_cache.emplace(key, b).first;
          }
          if (it != perm_cache.end() &&
              block_copy(dst, Ld, static_cast<const T*>(it->second.p), Lt.c_str(), alpha, beta))
            return;
        }
      }
    }
    scatter_permute(dst, Ld, src, Ls, alpha, beta, anti);
  }

  // the general case: the tiled permute kernel (any letter orders, the
  // antisymmetriser, broadcast letters); not recorded on the tape
  void scatter_permute(T* dst, const char* Ld, const T* src, const char* Ls, double alpha, double beta,
                       const char* anti) {
    ScatDesc d{};
    d.nd = static_cast<int>(strlen(Ld));
    auto ss = strides_of(Ls);
    d.total = 1;
    for (int k = 0; k < d.nd; ++k) {
      d.dim[k] = dimof(Ld[k]);
      d.total *= d.dim[k];
      const char* q = strchr(Ls, Ld[k]);
      d.sst[k] = q ? ss[q - Ls] : 0;
    }
    d.nswap = 0;
    for (const char* q = anti; *q; q += 2) {
      const char* pa = strchr(Ld, q[0]);
      const char* pb = strchr(Ld, q[1]);
      if (!pa || !pb) throw Fail{FTCC_ERR_STATE, "bad antisymmetriser"};
      d.sw[d.nswap][0] = static_cast<int>(pa - Ld);
      d.sw[d.nswap][1] = static_cast<int>(pb - Ld);
      d.nswap++;
    }
    const double reads = (d.nswap == 0 ? 1 : (d.nswap == 1 ? 2 : 4)) + (beta != 0.0 ? 1 : 0);
    timed_launch(kClsScatter, static_cast<double>(d.total) * (reads + 1) * sizeof(T), 0.0,
                 [&] { CU(launch_scatter<T>(src, dst, d, alpha, beta, st())); });
  }

  void pack(const T* src, const char* Ls, const std::string& rows, const std::string& cols, long long cpad, T* dst,
            void* hi, void* lo) {
    PackDesc d{};
    auto ss = strides_of(Ls);
    d.nr = static_cast<int>(rows.size());
    d.nc = static_cast<int>(cols.size());
    d.rows = 1;
    d.creal = 1;
    for (int k = 0; k < d.nr; ++k) {
      d.rdim[k] = dimof(rows[k]);
      d.rst[k] = ss[strchr(Ls, rows[k]) - Ls];
      d.rows *= d.rdim[k];
    }
    for (int k = 0; k < d.nc; ++k) {
      d.cdim[k] = dimof(cols[k]);
      d.cst[k] = ss[strchr(Ls, cols[k]) - Ls];
      d.creal *= d.cdim[k];
    }
    d.cpad = cpad;
    const double pbytes = static_cast<double>(d.rows) * (d.creal * sizeof(T) + d.cpad * (hi ? 4 : sizeof(T)));
    // rows already in GEMM order: a row split (bf16 halves) or a pitched copy
    if (rows + cols == std::string(Ls)) {
      timed_launch(kClsPack, pbytes, 0.0, [&] {
        if (hi)
          CU(launch_split_rows(reinterpret_cast<const float*>(src), d.creal, hi, lo, d.cpad, d.rows, d.creal, st()));
        else
          CU(cudaMemcpy2DAsync(dst, d.cpad * sizeof(T), src, d.creal * sizeof(T), d.creal * sizeof(T), d.rows,
                               cudaMemcpyDeviceToDevice, st()));
      });
      return;
    }
    timed_launch(kClsPack, pbytes, 0.0, [&] {
      if (hi) {
        CU(launch_pack_bf16x2(reinterpret_cast<const float*>(src), hi, lo, d, st()));
      } else {
        CU(launch_pack<T>(src, dst, d, st()));
      }
    });
  }

  // One GEMM operand: [rows][ld] row-major with K = cols contiguous.  Uses
  // the tensor in place when it already has that layout, a cached pack for
  // fixed operands, or packs into the scratch buffers (buf, buf2).
  struct Operand {
    const void* p;
    const void* p2;
    long long ld;
  };
  // Packs of the S-kernel inputs (t1, t2 of the current pass), kept for the
  // rest of the pass: t2 enters two contractions in the same packed order.
  struct AmpPack {
    const void* src;
    std::string L, rows, cols;
    long long ld;
    int kind;
    Buf a, b;
    bool valid;
  };
  std::vector<AmpPack> amp_cache;
  const void* amp_in[2] = {nullptr, nullptr};
  void amp_begin(const void* t1c, const void* t2c) {
    amp_in[0] = t1c;
    amp_in[1] = t2c;
    for (auto& e : amp_cache) e.valid = false;
  }
  void amp_end() { amp_in[0] = amp_in[1] = nullptr; }

  Operand operand(Tn<const T> X, const std::string& rows, const std::string& cols, long long k, int kind, Buf& buf,
                  Buf& buf2) {
    const long long q = kind == GEMM_TF32 ? 4 : (kind == GEMM_BF16X3 ? 8 : 1);
    const long long ld = (k + q - 1) / q * q;
    if (kind != GEMM_BF16X3 && rows + cols == std::string(X.L) && ld == k &&
        (kind != GEMM_TF32 || (reinterpret_cast<uintptr_t>(X.p) & 15) == 0))
      return {X.p, nullptr, k};
    long long nrow = 1;
    for (char ch : rows) nrow *= dimof(ch);
    const size_t es = kind == GEMM_BF16X3 ? 2 : sizeof(T);
    const size_t bytes = static_cast<size_t>(nrow) * ld * es;
    if (!X.fixed && X.p && (X.p == amp_in[0] || X.p == amp_in[1])) {
      AmpPack* slot = nullptr;
      for (auto& e : amp_cache) {
        if (e.rows == rows && e.cols == cols && e.ld == ld && e.kind == kind) {
          if (e.valid && e.src == X.p && e.L == X.L) return {e.a.p, e.b.p, ld};
          if (!e.valid && !slot) slot = &e;
        }
      }
      if (!slot) {
        amp_cache.push_back(AmpPack{nullptr, "", rows, cols, ld, kind, Buf{}, Buf{}, false});
        slot = &amp_cache.back();
      }
      ensure(h_, slot->a, bytes);
      if (kind == GEMM_BF16X3) {
        ensure(h_, slot->b, bytes);
        pack(X.p, X.L, rows, cols, ld, nullptr, slot->a.p, slot->b.p);
      } else {
        pack(X.p, X.L, rows, cols, ld, static_cast<T*>(slot->a.p), nullptr, nullptr);
      }
      slot->src = X.p;
      slot->L = X.L;
      slot->valid = true;
      return {slot->a.p, slot->b.p, ld};
    }
    if (X.fixed) {
      PackKey key{X.p, rows, cols, ld, kind};
      auto it = packed.find(key);
      if (it == packed.end()) {
        std::pair<Buf, Buf> bb;
        ensure(h_, bb.first, bytes);
        if (kind == GEMM_BF16X3) ensure(h_, bb.second, bytes);
        pack(X.p, X.L, rows, cols, ld, static_cast<T*>(bb.first.p), kind == GEMM_BF16X3 ? bb.first.p : nullptr,
             bb.second.p);
        it = packed.emplace(key, bb).first;
      }
      return {it->second.first.p, it->second.second.p, ld};
    }
    ensure(h_, buf, bytes);
    if (kind == GEMM_BF16X3) {
      ensure(h_, buf2, bytes);
      pack(X.p, X.L, rows, cols, ld, nullptr, buf.p, buf2.p);
    } else {
      pack(X.p, X.L, rows, cols, ld, static_cast<T*>(buf.p), nullptr, nullptr);
    }
    return {buf.p, buf2.p, ld};
  }

  // C(Lc) = beta_acc * C + alpha * P(sum over shared letters A(La) B(Lb))
  //
  // Among the 16 ways to feed this contraction to the GEMM (which operand is
  // "A", and the order of the row letters of each operand and of the summed
  // letters) the engine takes the one that moves the fewest bytes: an operand
  // already stored as [rows][K] is used in place, a fixed operand's pack is
  // cached, and a GEMM output already in C's layout (no antisymmetriser) is
  // written straight into C.
  void contract(Tn<T> C, double alpha, Tn<const T> A, Tn<const T> B, const char* anti = "", double beta_acc = 1.0) {
    if (recording) tape.push_back(Op{0, C.p, C.L, A.p, A.L, B.p, B.L, nullptr, alpha, beta_acc, anti});
    const std::string Lc = C.L;
    for (char ch : Lc)
      if (!strchr(A.L, ch) && !strchr(B.L, ch)) throw Fail{FTCC_ERR_STATE, "letter of C in neither operand"};
    for (const char* q = A.L; *q; ++q)
      if (!strchr(C.L, *q) && !strchr(B.L, *q)) throw Fail{FTCC_ERR_STATE, "free letter in A"};
    for (const char* q = B.L; *q; ++q)
      if (!strchr(C.L, *q) && !strchr(A.L, *q)) throw Fail{FTCC_ERR_STATE, "free letter in B"};
    auto size_of_letters = [&](const std::string& L) {
      long long s = 1;
      for (char ch : L) s *= dimof(ch);
      return s;
    };
    auto ordered = [](const std::string& from, const std::string& keep) {
      std::string out;
      for (char ch : from)
        if (keep.find(ch) != std::string::npos) out += ch;
      return out;
    };
    struct Plan {
      bool swap;
      std::string bat, Ml, Nl, Kl;
      bool direct, trans;
      long long cost;
    };
    Plan best{};
    best.cost = -1;
    const bool anti_none = anti[0] == 0;
    const long long csize = size_of_letters(Lc);
    for (int mask = 0; mask < 16; ++mask) {
      const bool swap = mask & 1;
      const Tn<const T>& X = swap ? B : A;
      const Tn<const T>& Y = swap ? A : B;
      const std::string LX = X.L, LY = Y.L;
      std::string bat, Mset, Nset, Kset;
      for (char ch : Lc) {
        const bool ix = LX.find(ch) != std::string::npos, iy = LY.find(ch) != std::string::npos;
        if (ix && iy) bat += ch;
        else if (ix) Mset += ch;
        else Nset += ch;
      }
      for (char ch : LX)
        if (Lc.find(ch) == std::string::npos) Kset += ch;
      const std::string Ml = (mask & 2) ? ordered(LX, Mset) : Mset;
      const std::string Nl = (mask & 4) ? ordered(LY, Nset) : Nset;
      const std::string Kl = (mask & 8) ? ordered(LY, Kset) : Kset;
      // the GEMM writes C in place when C's layout is [bat][M][N], or [bat][N][M]
      // with the output stored transposed
      const bool dn = anti_none && bat + Ml + Nl == Lc;
      const bool dt = anti_none && !dn && bat + Nl + Ml == Lc;
      const bool direct = dn || dt;
      long long cost = direct ? 0 : 2 * csize;
      if (!X.fixed && LX != bat + Ml + Kl) cost += 2 * size_of_letters(LX);
      if (!Y.fixed && LY != bat + Nl + Kl) cost += 2 * size_of_letters(LY);
      // the tensor-core tile is 128 rows high: a plan that puts fewer than 64
      // rows on M while N has more would run on the SIMT kernel instead
      if (gk != GEMM_F64 && size_of_letters(Mset) < 64 && size_of_letters(Nset) >= 64) cost += 4 * csize;
      if (best.cost < 0 || cost < best.cost) best = Plan{swap, bat, Ml, Nl, Kl, direct, dt, cost};
    }
    const Tn<const T>& GA = best.swap ? B : A;
    const Tn<const T>& GB = best.swap ? A : B;
    const std::string bat = best.bat, Ml = best.Ml, Nl = best.Nl, Kl = best.Kl;
    long long nb = 1, m = 1, n = 1, k = 1;
    for (char ch : bat) nb *= dimof(ch);
    for (char ch : Ml) m *= dimof(ch);
    for (char ch : Nl) n *= dimof(ch);
    for (char ch : Kl) k *= dimof(ch);
    if (nb * m * n == 0) return;
    if (counting) gemm_flops += 2 * nb * m * n * k;
    // N and K of at most 32 (t1- and F-sized operands): one thread per output row;
    // otherwise tensor cores when M fills half a tile
    const bool skinny = n <= 32 && k <= 32 && nb <= 65535;
    const bool tc = !skinny && (gk != GEMM_F64) && m >= 64 && k >= 8;   // narrow N uses a narrow tile
    const int kind = tc ? gk : (gk == GEMM_F64 ? GEMM_F64 : -1);   // -1: FP32 SIMT
    const Operand oa = operand(GA, bat + Ml, Kl, k, kind, pA, pA2);
    const Operand ob = operand(GB, bat + Nl, Kl, k, kind, pB, pB2);
    const std::string Lt = bat + Ml + Nl;
    const bool direct = best.direct;   // GEMM output is already C's layout
    if (!direct) ensure(h_, Ct, nb * m * n * sizeof(T));
    GemmArgs g{};
    g.batch = static_cast<int>(nb);
    g.M = static_cast<int>(m);
    g.N = static_cast<int>(n);
    g.K = static_cast<int>(k);
    g.A = oa.p;
    g.lda = oa.ld;
    g.sa = nb > 1 ? m * oa.ld : 0;
    g.B = ob.p;
    g.ldb = ob.ld;
    g.sb = nb > 1 ? n * ob.ld : 0;
    g.A2 = oa.p2;
    g.B2 = ob.p2;
    g.C = direct ? static_cast<void*>(C.p) : Ct.p;
    g.trans = best.trans ? 1 : 0;
    g.ldc = best.trans ? m : n;
    g.sc = m * n;
    g.alpha = direct ? alpha : 1.0;
    g.beta = direct ? beta_acc : 0.0;
    ensure(h_, skw, 64u << 20);   // split-K partials (SIMT and tensor-core kernels)
    g.work = skw.p;
    g.work_bytes = skw.bytes;
    if (kind == GEMM_TF32 || kind == GEMM_BF16X3) tune_tc(kind, g, nb * m * n * sizeof(T));
    const double es = kind == GEMM_BF16X3 ? 4.0 : static_cast<double>(sizeof(T));   // hi + lo halves
    const double gbytes = static_cast<double>(nb) * ((m + n) * k * es + m * n * sizeof(T) * (g.beta != 0.0 ? 2 : 1));
    const double gflops = 2.0 * nb * m * n * k;
    timed_launch(kind == GEMM_TF32 || kind == GEMM_BF16X3 ? kClsGemmTc : kClsGemmSimt, gbytes, gflops, [&] {
      if (skinny) CU(kind == GEMM_F64 ? gemm_skinny_f64(g, st()) : gemm_skinny_f32(g, st()));
      else if (kind == GEMM_F64) CU(gemm_f64(g, st()));
      else if (kind == -1) CU(gemm_f32(g, st()));
      else CU(gemm_tc(kind, g, h_->dev_err, st()));
    });
    if (!direct) {
      const bool rec = recording;   // part of this contraction, not an op of its own
      recording = false;
      scatter(C.p, C.L, static_cast<const T*>(Ct.p), Lt.c_str(), alpha, beta_acc, anti);
      recording = rec;
    }
  }

  // Tile-width / split-K autotuner for the tensor-core GEMM.  The first time
  // a shape (kind, batch, M, N, K, output order, accumulate or not) is met
  // outside a stream capture, every candidate (tile width 32 / 64 / 128 / 256
  // columns x built-in or no K split) runs on a scratch output, timed as a
  // plain launch (long products) or a graph replay of three launches (short
  // ones), and the fastest is kept for that shape; later calls (and the
  // captured graph) use it.  Shapes whose output exceeds 512 MB or whose work
  // exceeds 2 TFLOP keep the built-in choice, where the tile shape matters
  // least and a trial run costs the most.  The table lives in the home
  // context (ftcc_ctx::tuned), so later solves there reuse the choices.
  Buf tuneC;
  void tune_tc(int kind, GemmArgs& g, size_t out_bytes) {
    if (!b->opt.autotune) return;
    const std::array<int, 7> key{kind, g.batch, g.M, g.N, g.K, g.trans, g.beta != 0.0 ? 1 : 0};
    auto& tuned = h_->tuned;
    auto it = tuned.find(key);
    if (it != tuned.end()) {
      g.bn = it->second.first;
      g.split = it->second.second;
      return;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(st(), &cs));
    const double flops = 2.0 * g.batch * static_cast<double>(g.M) * g.N * g.K;
    if (cs != cudaStreamCaptureStatusNone || out_bytes > (512u << 20) || flops > 2e12) return;
    ensure(h_, tuneC, out_bytes);
    CU(cudaMemsetAsync(tuneC.p, 0, out_bytes, st()));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    GemmArgs t = g;
    t.C = tuneC.p;
    float best = -1.0f;
    std::pair<int, int> pick{0, 0};
    for (int bn : {32, 64, 128, 256}) {
      if (bn > 32 && g.N <= bn / 2) continue;   // mostly empty tiles
      for (int split : {0, 1}) {
        t.bn = bn;
        t.split = split;
        // device time alone.  A plain launch first (attributes, module load);
        // when it already runs for more than half a millisecond, host work
        // per launch is negligible and a second plain launch is the timing.
        // Shorter products are timed as a graph replay of three launches
        // captured once, so that host work per launch (tensor-map encoding,
        // the split-K reduction's launch) is not counted.
        constexpr int kReps = 3;
        float ms = 0.0f;
        CU(cudaEventRecord(e0, st()));
        CU(gemm_tc(kind, t, h_->dev_err, st()));
        CU(cudaEventRecord(e1, st()));
        CU(cudaEventSynchronize(e1));
        CU(cudaEventElapsedTime(&ms, e0, e1));
        if (ms > 0.5f) {
          CU(cudaEventRecord(e0, st()));
          CU(gemm_tc(kind, t, h_->dev_err, st()));
          CU(cudaEventRecord(e1, st()));
          CU(cudaEventSynchronize(e1));
          CU(cudaEventElapsedTime(&ms, e0, e1));
          if (best < 0.0f || ms < best) {
            best = ms;
            pick = {bn, split};
          }
          continue;
        }
        cudaGraph_t gr = nullptr;
        CU(cudaStreamBeginCapture(st(), cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = cudaSuccess;
        for (int rep = 0; rep < kReps && ce == cudaSuccess; ++rep) ce = gemm_tc(kind, t, h_->dev_err, st());
        const cudaError_t ee = cudaStreamEndCapture(st(), &gr);
        CU(ce);
        CU(ee);
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ge, gr, 0);
        cudaGraphDestroy(gr);
        CU(ie);
        cudaError_t re = cudaGraphLaunch(ge, st());   // upload and warm
        if (re == cudaSuccess) re = cudaEventRecord(e0, st());
        if (re == cudaSuccess) re = cudaGraphLaunch(ge, st());
        if (re == cudaSuccess) re = cudaEventRecord(e1, st());
        if (re == cudaSuccess) re = cudaEventSynchronize(e1);
        if (re == cudaSuccess) re = cudaEventElapsedTime(&ms, e0, e1);
        cudaGraphExecDestroy(ge);
        CU(re);
        ms /= kReps;
        if (best < 0.0f || ms < best) {
          best = ms;
          pick = {bn, split};
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tuned[key] = pick;
    g.bn = pick.first;
    g.split = pick.second;
  }

  void alloc_chunk() {
    const long long o = no, v = nv, x = static_cast<long long>(nxc) * nz;
    ensure(h_, ta, x * o * o * v * v * sizeof(T));
    ensure(h_, X, x * o * o * v * v * sizeof(T));
    ensure(h_, Wmnij, x * o * o * o * o * sizeof(T));
    ensure(h_, Wabef, x * v * v * v * v * sizeof(T));
    ensure(h_, Wmbej, x * o * v * v * o * sizeof(T));
    ensure(h_, Y, x * o * o * v * o * sizeof(T));
    ensure(h_, Fae, x * v * v * sizeof(T));
    ensure(h_, Fmi, x * o * o * sizeof(T));
    ensure(h_, Fme, x * o * v * sizeof(T));
    ensure(h_, Ft, x * v * v * sizeof(T));
    ensure(h_, Ft2, x * o * o * sizeof(T));
    ensure(h_, R, x * o * o * v * v * sizeof(T));
    ensure(h_, R2, x * o * o * v * v * sizeof(T));
    const long long po = o * (o - 1) / 2, pv = v * (v - 1) / 2;
    ensure(h_, tp, std::max(1LL, x * po * pv) * sizeof(T));
    ensure(h_, WAmn, std::max(1LL, x * po * po) * sizeof(T));
    ensure(h_, WAef, std::max(1LL, x * pv * pv) * sizeof(T));
    ensure(h_, Lp, std::max(1LL, x * po * pv) * sizeof(T));
    if (!pairsO.p) {
      auto table = [&](Buf& b, long long n) {
        std::vector<int2> t;
        for (int p = 0; p < n; ++p)
          for (int q = p + 1; q < n; ++q) t.push_back(make_int2(p, q));
        ensure(h_, b, std::max<size_t>(1, t.size()) * sizeof(int2));
        if (!t.empty()) {
          CU(cudaMemcpyAsync(b.p, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice, st()));
          CU(cudaStreamSynchronize(st()));
        }
      };
      table(pairsO, o);
      table(pairsV, v);
    }
  }

  // Workspaces of the block-sparse S kernel for nxc tau points: the
  // amplitude-derived operands (ta = tau, tt = tau in [a][b][m] order, Y =
  // s2 in ring order, X = the W_mbej operand), the intermediates W'_mnij,
  // W'_abef, W_mbej (ring order) and R, the vector intermediates, and the
  // <mn||ef> block in the W_mbej operand order.
  void sparse_alloc() {
    const long long n = no, n3 = n * n * n, x = nxc;
    // R2: the ring term [i][a][b]; Lp: the ladders at the canonical elements [i][j][a]
    for (Buf* q : {&ta, &tt, &Y, &X, &Wmnij, &Wabef, &Wmbej, &R, &R2, &Lp}) ensure(h_, *q, x * n3 * sizeof(T));
    for (Buf* q : {&Fme, &Fae, &Fmi, &Ft, &Ft2}) ensure(h_, *q, x * n * sizeof(T));
    ensure(h_, Vp, n3 * sizeof(T));
    // cotangents of the transpose (sparse_vjp)
    for (Buf* q : {&bR, &bta, &btt, &bY, &bX, &bWmnij, &bWabef, &bWmbej}) ensure(h_, *q, x * n3 * sizeof(T));
    for (Buf* q : {&bFme, &bFae, &bFmi, &bFt, &bFt2}) ensure(h_, *q, x * n * sizeof(T));
    ensure(h_, bP, n3 * sizeof(T));
    CU(launch_sp_swap12<T>(V("zmnef"), no, static_cast<T*>(Vp.p), st()));
  }

  SpBlocksT<T> sp_blocks() {
    return SpBlocksT<T>{V("zmnef"), V("zmbef"), V("zmnie"), V("zmnij"), V("zabef"), V("zmbej"),
                        V("zmnej"), V("zmaie"), V("zabij"), V("zabej"), V("zmbij")};
  }

  void sector_product(const SecTab& tab, const T* A, long long ax, const T* Bm, long long bx, T* C, double alpha,
                      int swapB, long long s0, long long s1, long long s2, long long s3, const T* A2 = nullptr,
                      const T* B2 = nullptr, int anti4 = 0, int store = 0) {
    {
      const long long n3 = static_cast<long long>(no) * no * no;
      SecGemmArgsT<T> g{};
      g.A = A;
      g.ax = ax;
      g.B = Bm;
      g.bx = bx;
      g.C = C;
      g.cx = n3;
      g.alpha = alpha;
      g.n = no;
      g.swapB = swapB;
      g.s0 = s0;
      g.s1 = s1;
      g.s2 = s2;
      g.s3 = s3;
      g.ent = static_cast<const int2*>(tab.ent.p);
      g.kl = static_cast<const int*>(tab.kl.p);
      g.sec = static_cast<const int4*>(tab.sec.p);
      g.work = static_cast<const int4*>(tab.work.p);
      g.A2 = A2;
      g.B2 = B2;
      g.anti4 = anti4;
      g.store = store;
      const double fl = tab.flops * nx * (A2 ? 2 : 1);
      if (counting) gemm_flops += static_cast<long long>(fl);
      timed_launch(kClsSector, static_cast<double>(nx) * n3 * (A2 ? 5 : 3) * sizeof(T), fl, [&] {
        // (one stream: running the small sectors beside the large ones on a
        // side stream measured 3.81 -> 3.86 ms per FP64 iteration of the
        // 114-orbital gas, no gain in FP32; it pays in the transpose, below)
        CU(launch_sector_gemm<T>(g, tab.nwork, nx, st()));
        SecGemmArgsT<T> gs = g;
        gs.work = static_cast<const int4*>(tab.work_small.p);
        CU(launch_sector_gemm_small<T>(gs, tab.nwork_small, nx, st()));
      });
    }
  }

  // The block-sparse S kernel: the same terms as s_kernel (Eqs. ccS1/ccS2
  // through the same intermediates) with s1 and every two-index factor
  // diagonal and the four-index factors in N^3 storage; the five products
  // of two four-index factors (W_mnij's tau term, W_mbej's X term, the two
  // ladders and the ring) run over pair-charge sectors.
  //
  // Outside the transpose's recomputation (pairs = true) W_mnij's tau term
  // and both ladders run over unordered pairs (i < j, m < n, e < f, a < b):
  // with W'_mnij and W'_abef antisymmetrised (their s1 terms become the
  // P(ij) / P(ab) forms), W^A_ijmn = W'^A_ijmn + sum_{e<f} tau_ij^ef <mn||ef>
  // and L_ij^ab = sum_{m<n} W^A_ijmn tau_mn^ab + sum_{e<f} tau_ij^ef W'^A_abef
  // give P(ij)P(ab) of the two ladders, added to R as L/4 in its four
  // orientations (R enters S2 through P(ij)P(ab)); each product is an eighth
  // of its ordered form.  The transpose recomputes the ordered form.
  void sparse_s_kernel(const T* t1c, const T* t2c, T* S1c, T* S2c, int nxcur, bool pairs = true) {
    vjp_fwd_key = nullptr;
    {
      nx = nxcur;
      const int n = no;
      const long long n2 = static_cast<long long>(n) * n, n3 = n2 * n;
      const int16_t* imp = static_cast<const int16_t*>(b->imp.p);
      T *pta = (T*)ta.p, *ptp = (T*)tt.p, *ptr = (T*)Y.p, *pxp = (T*)X.p, *pw1 = (T*)Wmnij.p, *pwab = (T*)Wabef.p,
        *pwr = (T*)Wmbej.p, *pR = (T*)R.p, *pXr = (T*)R2.p;
      const SpBlocksT<T> VB = sp_blocks();
      const double slice = static_cast<double>(nx) * n3 * sizeof(T);
      timed_launch(kClsOther, 6 * slice, 0.0,
                   [&] {
                     CU(launch_sp_amp<T>(t1c, t2c, imp, n, nx, pta, ptp, ptr, pxp, pairs ? 1 : 0,
                                         pairs ? static_cast<const int*>(b->vswap.p) : nullptr, b->nvswap, st()));
                   });
      SpVecArgsT<T> v{};
      v.t1 = t1c;
      v.t2 = t2c;
      v.fov = F("zme");
      v.foo = F("zmi");
      v.fvv = F("zae");
      v.fvo = F("zai");
      v.Voovv = VB.oovv;
      v.Vovvv = VB.ovvv;
      v.Vooov = VB.ooov;
      v.Vovov = VB.ovov;
      v.Voovo = VB.oovo;
      v.imp = imp;
      v.l1 = static_cast<const int*>(b->vl1.p);
      v.off1 = static_cast<const int*>(b->voff1.p);
      v.l2 = static_cast<const int*>(b->vl2.p);
      v.off2 = static_cast<const int*>(b->voff2.p);
      v.n = n;
      v.Fme = (T*)Fme.p;
      v.Fae = (T*)Fae.p;
      v.Fmi = (T*)Fmi.p;
      v.S1 = S1c;
      v.Ft = (T*)Ft.p;
      v.Ft2 = (T*)Ft2.p;
      timed_launch(kClsOther, 6 * slice, 0.0, [&] { CU(launch_sp_vectors<T>(v, nx, st())); });
      timed_launch(kClsScatter, 3 * slice + 6.0 * n3 * sizeof(T), 0.0,
                   [&] {
                     CU(launch_sp_wbase<T>(t1c, VB, imp, n, nx, pw1, pwab, pwr, pairs ? 1 : 0,
                                           pairs ? static_cast<const int*>(b->vrot.p) : nullptr, b->nvrot, st()));
                   });
      const int* canon = static_cast<const int*>(b->canon.p);
      const int ncanon = static_cast<int>(b->ncanon);
      if (pairs)
        timed_launch(kClsScatter, 4.0 * nx * ncanon * 4 * sizeof(T), 0.0, [&] {
          CU(launch_sp_canon<T>(t1c, t2c, VB, imp, canon, ncanon, n, nx, pta, ptp, pw1, pwab, st()));
        });
      // W'_mnij += 1/2 tau_ij^ef <mn||ef>        rows (i,j) | (m,n) by q_i + q_j, sum over e
      // (unordered: W^A_ijmn += sum_{e<f} tau_ij^ef <mn||ef> for i < j, m < n)
      if (pairs) sector_product(b->ssum_u, pta, n3, VB.oovv, 0, pw1, 1.0, 0, n2, n, 1, 0);
      else sector_product(b->ssum, pta, n3, VB.oovv, 0, pw1, 0.5, 0, n2, n, 1, 0);
      // W_mbej -= X_jn^fb <mn||ef>                rows (j,b) | (m,e) by q_j - q_b, sum over n
      sector_product(b->sdiff, pxp, n3, static_cast<const T*>(Vp.p), 0, pwr, -1.0, 0, n2, n, 1, 0);
      timed_launch(kClsScatter, 5 * slice, 0.0, [&] {
        CU(launch_sp_rinit<T>(t1c, t2c, (T*)Ft.p, (T*)Ft2.p, VB, imp, static_cast<const int*>(b->vall.p), b->nvall, n,
                              nx, pR, st()));
      });
      T* pLc = pairs ? (T*)Lp.p : nullptr;
      if (pairs) {
        // both ladders L at the canonical elements only, rows i < j | a < b,
        // sums over m < n and e < f: stored at Lc[i][j][a] (written once) and
        // added by the S2 kernel, which works on the canonical elements (as
        // L/4 in the four orientations of R it was four read-modify-writes)
        sector_product(b->ssum_u, pw1, n3, ptp, n3, pLc, 1.0, 0, n2, n, 1, 0, pta, pwab, 0, 1);
      } else {
        // hole ladder 1/8 W'_ijmn tau_mn^ab          rows (i,j) | (a,b) by q_i + q_j, sum over m
        sector_product(b->ssum, pw1, n3, ptp, n3, pR, 0.125, 0, n2, n, 1, 0);
        // particle ladder 1/8 tau_ij^ef W'_abef      rows (i,j) | (a,b), sum over e
        sector_product(b->ssum, pta, n3, pwab, n3, pR, 0.125, 0, n2, n, 1, 0);
      }
      // ring s_im^ae W_mbej                        rows (i,a) | (j,b) by q_i - q_a, sum over m
      // ring: rows (i, a), columns (b, j) (wr rows swapped); stored apart as
      // Xr[i][a][b] (each position written once, nearly contiguous along a
      // CTA's columns), added into S2 by its gather; into R[i][j][a] it would
      // be a read-modify-write of one 32-byte sector per output
      sector_product(b->sdiff, ptr, n3, pwr, n3, pXr, 1.0, 1, n2, n, 1, 0, nullptr, nullptr, 0, 1);
      timed_launch(kClsScatter, 6 * slice, 0.0,
                   [&] { CU(launch_sp_s2<T>(pR, pXr, pLc, VB.vvoo, imp, canon, ncanon, n, nx, S2c, st())); });
    }
  }

  // One transposed sector product (see SecTnArgs): with fixed D (dx = 0)
  // the slices are summed inside the kernel.
  void sector_tn(const SecTab& tab, double* D, long long dx, const double* G, const double* A, long long ax,
                 double alpha, int swapD, int swapA, long long g0, long long g1, long long g2, long long g3,
                 int antiA = 0, int anti4 = 0) {
    const long long n3 = static_cast<long long>(no) * no * no;
    SecTnArgs g{};
    g.D = D;
    g.dx = dx;
    g.G = G;
    g.gx = n3;
    g.A = A;
    g.ax = ax;
    g.alpha = alpha;
    g.n = no;
    g.nx = nx;
    g.swapD = swapD;
    g.swapA = swapA;
    g.g0 = g0;
    g.g1 = g1;
    g.g2 = g2;
    g.g3 = g3;
    g.ent = static_cast<const int2*>(tab.ent.p);
    g.kl = static_cast<const int*>(tab.kl.p);
    g.sec = static_cast<const int4*>(tab.sec.p);
    g.work = static_cast<const int4*>(tab.work.p);
    g.antiA = antiA;
    g.anti4 = anti4;
    timed_launch(kClsSector, static_cast<double>(nx) * n3 * 3 * sizeof(double), tab.flops * nx, [&] {
      // the sectors of at most 16 pairs (latency-bound, short K loops) run on
      // the side stream beside the large ones: the two write disjoint outputs
      // (kept on one stream for dx = 0, where the output is one fixed block);
      // the adjoint of the 114-orbital gas 0.114 -> 0.108 s
      SecTnArgs gs = g;
      gs.work = static_cast<const int4*>(tab.work_small.p);
      const bool fork = dx != 0 && tab.nwork > 0 && tab.nwork_small > 0;
      if (fork) CU(launch_sector_tn_small(gs, tab.nwork_small, side_begin()));
      CU(launch_sector_tn(g, tab.nwork, st()));
      if (fork) side_end();
      else CU(launch_sector_tn_small(gs, tab.nwork_small, st()));
    });
  }

  // Transpose of sparse_s_kernel: (u1, u2) = cotangents of (S1, S2) ->
  // (t1bar, t2bar) = cotangents of (s1, s2); with want_fixed_bar the
  // cotangents of the integral and Fock blocks accumulate in fixed_bar.
  // The forward intermediates are recomputed first (S lands in t1bar /
  // t2bar and is overwritten).  Each product C += alpha A B of the forward
  // pass gives Abar += alpha Cbar B and Bbar += alpha Cbar^T A.
  void sparse_vjp(const T* t1c, const T* t2c, const T* u1, const T* u2, T* t1bar, T* t2bar, int nxcur) {
    if constexpr (sizeof(T) == 8) {
      // the forward intermediates (ordered ladders), recomputed unless the
      // lambda sweep's fixed amplitudes already left them in place
      nx = nxcur;
      if (!(vjp_fwd_reuse && vjp_fwd_key == t2c && vjp_fwd_nx == nxcur)) {
        sparse_s_kernel(t1c, t2c, t1bar, t2bar, nxcur, false);
        if (vjp_fwd_reuse) {
          vjp_fwd_key = t2c;
          vjp_fwd_nx = nxcur;
        }
      }
      const int n = no;
      const long long n2 = static_cast<long long>(n) * n, n3 = n2 * n;
      const int16_t* imp = static_cast<const int16_t*>(b->imp.p);
      const SpBlocks VB = sp_blocks();
      double *Rb = (double*)bR.p, *tab_ = (double*)bta.p, *tpb = (double*)btt.p, *trb = (double*)bY.p,
             *xpb = (double*)bX.p, *w1b = (double*)bWmnij.p, *wabb = (double*)bWabef.p, *wrb = (double*)bWmbej.p;
      for (double* q : {tab_, tpb, trb, xpb, w1b, wabb, wrb})
        CU(cudaMemsetAsync(q, 0, nx * n3 * sizeof(double), st()));
      const double *ta_ = (double*)ta.p, *tp_ = (double*)tt.p, *tr_ = (double*)Y.p, *xp_ = (double*)X.p,
                   *w1_ = (double*)Wmnij.p, *wab_ = (double*)Wabef.p, *wr_ = (double*)Wmbej.p;
      const int* vall = static_cast<const int*>(b->vall.p);
      timed_launch(kClsScatter, 2.0 * nx * n3 * 8, 0.0,
                   [&] { CU(launch_sp_s2_t(u2, imp, vall, b->nvall, n, nx, Rb, st())); });
      // ring: R += tr wr (rows (i,a) | (j,b) swapped, output (n2, 1, 0, n))
      sector_tn(b->sdiff, trb, n3, Rb, wr_, n3, 1.0, 0, 1, n2, 1, 0, n);
      sector_tn(b->sdiff, wrb, n3, Rb, tr_, n3, 1.0, 1, 0, 0, n, n2, 1);
      // The ladders' cotangents over unordered pairs.  R-bar = P(ij)P(ab)
      // S2-bar is antisymmetric in ij and in ab, and so are the results
      // (tau, <mn||ef> antisymmetric in both pairs; W'_abef and W'_mnij in
      // their second pair): a sum over ordered (a, b) is twice the sum over
      // a < b of R-bar times the operand antisymmetrised in (a, b), and each
      // canonical output (i < j, e < f) is written to its four orientations.
      // particle ladder: R += 1/8 ta wab
      sector_tn(b->ssum_u, tab_, n3, Rb, wab_, n3, 0.25, 0, 0, n2, n, 1, 0, 1, 1);
      sector_tn(b->ssum_u, wabb, n3, Rb, ta_, n3, 0.25, 0, 0, 1, 0, n2, n, 0, 1);
      // hole ladder: R += 1/8 w1 tp
      sector_tn(b->ssum_u, w1b, n3, Rb, tp_, n3, 0.25, 0, 0, n2, n, 1, 0, 0, 1);
      sector_tn(b->ssum_u, tpb, n3, Rb, w1_, n3, 0.25, 0, 0, 1, 0, n2, n, 1, 1);
      // W_mbej: wr -= xp Vp;  W_mnij: w1 += 1/2 ta <mn||ef>
      sector_tn(b->sdiff, xpb, n3, wrb, static_cast<const double*>(Vp.p), 0, -1.0, 0, 0, n2, n, 1, 0);
      sector_tn(b->ssum_u, tab_, n3, w1b, VB.oovv, 0, 1.0, 0, 0, n2, n, 1, 0, 0, 1);
      double* Vbar[11] = {nullptr};
      double* fbar[4] = {nullptr};
      if (want_fixed_bar) {
        const char* eri_L[11] = {"zmnef", "zmbef", "zmnie", "zmnij", "zabef", "zmbej",
                                 "zmnej", "zmaie", "zabij", "zabej", "zmbij"};
        for (int k = 0; k < 11; ++k) Vbar[k] = fixed_adjoint(V(eri_L[k]));
        const char* f_L[4] = {"zme", "zae", "zmi", "zai"};
        for (int k = 0; k < 4; ++k) fbar[k] = fixed_adjoint(F(f_L[k]));
        double* Vpb = (double*)bP.p;
        CU(cudaMemsetAsync(Vpb, 0, n3 * sizeof(double), st()));
        sector_tn(b->sdiff, Vpb, 0, wrb, xp_, n3, -1.0, 0, 0, 1, 0, n2, n);
        CU(launch_sp_swap12_add(Vpb, n, Vbar[0], st()));
        sector_tn(b->ssum, Vbar[0], 0, w1b, ta_, n3, 0.5, 0, 0, 1, 0, n2, n);
      }
      SpVjpArgs va{};
      va.t1 = t1c;
      va.t2 = t2c;
      va.Ft = (double*)Ft.p;
      va.Ft2 = (double*)Ft2.p;
      va.Fme = (double*)Fme.p;
      va.Fae = (double*)Fae.p;
      va.Fmi = (double*)Fmi.p;
      va.S1b = u1;
      va.Rb = Rb;
      va.w1b = w1b;
      va.wabb = wabb;
      va.wrb = wrb;
      va.tab = tab_;
      va.tpb = tpb;
      va.trb = trb;
      va.xpb = xpb;
      va.V = VB;
      va.imp = imp;
      va.list = vall;
      va.nlist = b->nvall;
      va.l1 = static_cast<const int*>(b->vl1.p);
      va.off1 = static_cast<const int*>(b->voff1.p);
      va.l2 = static_cast<const int*>(b->vl2.p);
      va.off2 = static_cast<const int*>(b->voff2.p);
      va.n = n;
      va.Ftb = (double*)bFt.p;
      va.Ft2b = (double*)bFt2.p;
      va.Faeb = (double*)bFae.p;
      va.Fmib = (double*)bFmi.p;
      va.Fmeb = (double*)bFme.p;
      va.t1b = t1bar;
      va.t2b = t2bar;
      timed_launch(kClsOther, 12.0 * nx * n3 * 8, 0.0, [&] { CU(launch_sp_vjp_vectors(va, nx, st())); });
      timed_launch(kClsScatter, 12.0 * nx * n3 * 8, 0.0, [&] { CU(launch_sp_t2bar(va, nx, st())); });
      if (want_fixed_bar) CU(launch_sp_fixed_bar(va, u2, nullptr, Vbar, fbar, nx, st()));
    }
  }

  // dst[zx][P][Q] from a dense [zx][l0][l1][l2][l3] (dims d0 = d1, d2 = d3;
  // P over pairs of l0 < l1, Q over l2 < l3), the first pair antisymmetrised
  // on the way when anti
  void pair_pack(const T* src, T* dst, long long nb, bool first_hole, bool second_hole, bool anti) {
    const long long n1 = first_hole ? no : nv, n2 = second_hole ? no : nv;
    const long long np1 = n1 * (n1 - 1) / 2, np2 = n2 * (n2 - 1) / 2;
    const long long s3 = 1, s2 = n2, s1 = n2 * n2, s0 = n1 * n2 * n2, sb = n1 * n1 * n2 * n2;
    timed_launch(kClsPack, static_cast<double>(nb) * (sb + np1 * np2) * sizeof(T), 0.0, [&] {
      CU(launch_pair_pack<T>(src, dst, nb, sb, static_cast<const int2*>((first_hole ? pairsO : pairsV).p), np1,
                             static_cast<const int2*>((second_hole ? pairsO : pairsV).p), np2, s0, s1, s2, s3,
                             anti ? 1 : 0, 1.0, st()));
    });
  }

  // S kernel for nx tau slices of every instance (Eqs. ccS1 and ccS2
  // evaluated through the intermediates of the factorised CCSD equations;
  // the tau*<mn||ef> part of the particle-ladder intermediate is carried by
  // W_mnij with weight 1/2).  Inputs [z][x][...] with nx slices per instance.
  void s_kernel(const T* t1c, const T* t2c, T* S1c, T* S2c, int nxcur) {
    if (sp) {
      sparse_s_kernel(t1c, t2c, S1c, S2c, nxcur);
      return;
    }
    nx = nxcur;
    amp_begin(t1c, t2c);
    T *pta = (T*)ta.p, *pX = (T*)X.p, *pWmnij = (T*)Wmnij.p, *pWabef = (T*)Wabef.p,
      *pWmbej = (T*)Wmbej.p, *pY = (T*)Y.p, *pFae = (T*)Fae.p, *pFmi = (T*)Fmi.p, *pFme = (T*)Fme.p,
      *pFt = (T*)Ft.p, *pFt2 = (T*)Ft2.p, *pR = (T*)R.p, *pR2 = (T*)R2.p;
    using CT = Tn<const T>;
    auto CV = [this](const char* L) { return Tn<const T>{V(L), L, true}; };
    // tau = s2 + P(ij) s1 s1 and X = 1/2 s2 + s1 s1 in one pass over s2
    if (recording) {
      tape.push_back(Op{2, nullptr, "", t1c, "", t2c, "", pta, 0.5, 1.0, ""});
      tape.push_back(Op{3, pX, "", t1c, "", t2c, "", nullptr, 0.5, 1.0, ""});
    }
    timed_launch(kClsOther, 3.0 * nz * nx * no * no * nv * nv * sizeof(T), 0.0,
                 [&] { CU(launch_tau<T>(t1c, t2c, nullptr, pta, pX, 0.5, 1.0, nz * nx, no, nv, st())); });
    // F_me = f_me + sum_nf s_n^f <mn||ef>
    scatter(pFme, "zxme", F("zme"), "zme", 1.0, 0.0, "");
    contract({pFme, "zxme"}, 1.0, CT{t1c, "zxnf"}, CV("zmnef"));
    // The s1 s1 part of tau~ in F_ae and F_mi is -1/2 s_m^a (F_me - f_me) and
    // +1/2 s_i^e (F_me - f_me); with the f_me terms they combine to F_me, and
    // only s2 enters the quartic contractions (whose s2 pack the S1 term shares).
    // F_ae = f_ae - 1/2 s_m^a F_me + s_m^f <ma||fe> - 1/2 s_mn^af <mn||ef>
    scatter(pFae, "zxae", F("zae"), "zae", 1.0, 0.0, "");
    contract({pFae, "zxae"}, -0.5, CT{pFme, "zxme"}, CT{t1c, "zxma"});
    contract({pFae, "zxae"}, 1.0, CT{t1c, "zxmf"}, CV("zmafe"));
    contract({pFae, "zxaf"}, -0.5, CT{t2c, "zxmnae"}, CV("zmnfe"));
    // F_mi = f_mi + 1/2 s_i^e F_me + s_n^e <mn||ie> + 1/2 s_in^ef <mn||ef>
    scatter(pFmi, "zxmi", F("zmi"), "zmi", 1.0, 0.0, "");
    contract({pFmi, "zxmi"}, 0.5, CT{t1c, "zxie"}, CT{pFme, "zxme"});
    contract({pFmi, "zxmi"}, 1.0, CT{t1c, "zxne"}, CV("zmnie"));
    contract({pFmi, "zxmi"}, 0.5, CT{t2c, "zxinef"}, CV("zmnef"));
    // S2 is assembled as P(ij)P(ab) R + <ab||ij> with R = R1 + R2 (below).
    // A contribution X that is already antisymmetric in ij enters R as X/2
    // when the paper applies P(ab) to it (P(ij)P(ab) X = 2 P(ab) X), likewise
    // for ab, and a fully antisymmetric one as X/4.  A contribution may also
    // be relabelled, X -> -X(i<->j) or -X(a<->b), which P(ij)P(ab) maps to
    // the same result; the labels are chosen so that each GEMM writes its
    // accumulator in place.  The same argument lets an intermediate used only
    // inside such a term carry 2Z in place of P(ij)Z (W_mnij, W_abef).
    //
    // W'_mnij = <mn||ij> - 2 s_i^e <mn||je> + 1/2 ta_ij^ef <mn||ef>, stored [ij][mn]   [o^4 v^2]
    scatter(pWmnij, "zxijmn", V("zmnij"), "zmnij", 1.0, 0.0, "");
    contract({pWmnij, "zxijmn"}, -2.0, CT{t1c, "zxie"}, CV("zmnje"));
    // Outside the recorded (adjoint) pass the tau <mn||ef> term and both
    // ladders run over unordered pairs (below); the recorded pass keeps the
    // dense contractions, whose transposes the tape replays.
    const bool pairs = !recording && no >= 2 && nv >= 2;
    if (!pairs) contract({pWmnij, "zxijmn"}, 0.5, CT{pta, "zxijef"}, CV("zmnef"));
    // W'_abef = <ab||ef> - 2 s_m^a <mb||ef>
    scatter(pWabef, "zxabef", V("zabef"), "zabef", 1.0, 0.0, "");
    contract({pWabef, "zxabef"}, -2.0, CT{t1c, "zxma"}, CV("zmbef"));
    // W_mbej = <mb||ej> + s_j^f <mb||ef> - s_n^b <mn||ej> - (1/2 s_jn^fb + s_j^f s_n^b) <mn||ef>,
    // stored [jb][me] for the ring   [o^3 v^3]
    scatter(pWmbej, "zxjbme", V("zmbej"), "zmbej", 1.0, 0.0, "");
    contract({pWmbej, "zxjbme"}, 1.0, CT{t1c, "zxjf"}, CV("zmbef"));
    contract({pWmbej, "zxjbme"}, -1.0, CT{t1c, "zxnb"}, CV("zmnej"));
    contract({pWmbej, "zxjbme"}, -1.0, CT{pX, "zxjnfb"}, CV("zmnef"));
    // S1 (Eq. ccS1)
    scatter(S1c, "zxia", F("zai"), "zai", 1.0, 0.0, "");
    contract({S1c, "zxia"}, 1.0, CT{t1c, "zxie"}, CT{pFae, "zxae"});
    contract({S1c, "zxia"}, -1.0, CT{t1c, "zxma"}, CT{pFmi, "zxmi"});
    contract({S1c, "zxia"}, 1.0, CT{t2c, "zximae"}, CT{pFme, "zxme"});
    contract({S1c, "zxia"}, -1.0, CT{t1c, "zxnf"}, CV("znaif"));
    contract({S1c, "zxia"}, -0.5, CT{t2c, "zximef"}, CV("zmaef"));
    contract({S1c, "zxia"}, -0.5, CT{t2c, "zxmnae"}, CV("znmei"));
    // S2 (Eq. ccS2)
    scatter(pFt, "zxbe", pFae, "zxbe", 1.0, 0.0, "");
    contract({pFt, "zxbe"}, -0.5, CT{t1c, "zxmb"}, CT{pFme, "zxme"});
    scatter(pFt2, "zxmj", pFmi, "zxmj", 1.0, 0.0, "");
    contract({pFt2, "zxmj"}, 0.5, CT{t1c, "zxje"}, CT{pFme, "zxme"});
    // R1 [ij][ab]
    contract({pR, "zxijab"}, 0.5, CT{t2c, "zxijae"}, CT{pFt, "zxbe"}, "", 0.0);        // P(ab) s_ij^ae Ft_be
    contract({pR, "zxijab"}, 0.5, CT{pFt2, "zxmi"}, CT{t2c, "zxjmab"});                // -P(ij) s_im^ab Ft2_mj, i<->j
    if (!pairs) {
      contract({pR, "zxijab"}, 0.125, CT{pWmnij, "zxijmn"}, CT{pta, "zxmnab"});         // hole ladder
      contract({pR, "zxijab"}, 0.125, CT{pta, "zxijef"}, CT{pWabef, "zxabef"});         // particle ladder
    } else {
      // W^A_ijmn = (W'_ijmn - W'_jimn)/2 + sum_{e<f} tau_ij^ef <mn||ef> and
      // W^A_abef = (W'_abef - W'_baef)/2 are fully antisymmetric and give
      // P(ij)P(ab) of the two ladders above (the s1 terms of W' become their
      // P(ij) / P(ab) forms), i.e. the contribution
      //   L_ij^ab = sum_{m<n} W^A_ijmn tau_mn^ab + sum_{e<f} tau_ij^ef W^A_abef
      // to S2, computed for i<j, a<b and added to R as L/4 in every orientation
      // (R enters S2 through P(ij)P(ab)).  Each product is an eighth of the
      // dense one.
      T *ptp = (T*)tp.p, *pWAmn = (T*)WAmn.p, *pWAef = (T*)WAef.p, *pLp = (T*)Lp.p;
      const long long zx = static_cast<long long>(nz) * nx;
      if (!Vp.p) {
        const long long po = static_cast<long long>(no) * (no - 1) / 2, pv = static_cast<long long>(nv) * (nv - 1) / 2;
        ensure(h_, Vp, std::max(1LL, static_cast<long long>(nz) * po * pv) * sizeof(T));
        pair_pack(V("zmnef"), static_cast<T*>(Vp.p), nz, true, false, false);
      }
      pair_pack(pta, ptp, zx, true, false, false);
      pair_pack(pWmnij, pWAmn, zx, true, true, true);
      contract({pWAmn, "zxIJ"}, 1.0, CT{ptp, "zxIE"}, CT{static_cast<const T*>(Vp.p), "zJE", true});
      pair_pack(pWabef, pWAef, zx, false, false, true);
      contract({pLp, "zxIA"}, 1.0, CT{pWAmn, "zxIJ"}, CT{ptp, "zxJA"}, "", 0.0);
      contract({pLp, "zxIA"}, 1.0, CT{ptp, "zxIE"}, CT{pWAef, "zxAE"});
      timed_launch(kClsScatter, static_cast<double>(zx) * no * no * nv * nv * 2 * sizeof(T), 0.0,
                   [&] { CU(launch_pair_unpack_add<T>(pR, pLp, zx, no, nv, 0.25, st())); });
    }
    contract({pR, "zxijab"}, 0.5, CT{t1c, "zxie"}, CV("zabej"));                        // P(ij) s_i^e <ab||ej>
    contract({pR, "zxijab"}, -0.5, CT{t1c, "zxma"}, CV("zmbij"));                       // -P(ab) s_m^a <mb||ij>
    // R2 [ia][jb]
    contract({pR2, "zxiajb"}, 1.0, CT{t2c, "zximae"}, CT{pWmbej, "zxjbme"}, "", 0.0);  // ring
    contract({pY, "zxibjm"}, 1.0, CT{t1c, "zxie"}, CV("zmbej"), "", 0.0);              // Y_imbj = s_i^e <mb||ej>
    contract({pR2, "zxiajb"}, 1.0, CT{pY, "zxiajm"}, CT{t1c, "zxmb"});                 // -P(ij)P(ab) s_m^a Y_imbj, a<->b
    // S2 = P(ij)P(ab) (R + R2) + <ab||ij>: one pass over unordered index pairs
    if (recording) {
      tape.push_back(Op{1, S2c, "zxijab", pR, "zxijab", nullptr, "", nullptr, 1.0, 0.0, "ijab"});
      tape.push_back(Op{1, S2c, "zxijab", pR2, "zxiajb", nullptr, "", nullptr, 1.0, 1.0, "ijab"});
      tape.push_back(Op{1, S2c, "zxijab", V("zabij"), "zabij", nullptr, "", nullptr, 1.0, 1.0, ""});
    }
    {
      const long long o = no, v = nv;
      Anti4Desc d{};
      d.nzx = nz * nx;
      d.nx = nx;
      d.no = no;
      d.nv = nv;
      d.nsrc = 2;
      d.src[0] = AntiSrc{pR, o * o * v * v, o * v * v, v * v, v, 1, 1.0};     // [ij][ab]
      d.src[1] = AntiSrc{pR2, o * o * v * v, v * o * v, v, o * v, 1, 1.0};    // [ia][jb]
      d.vp = V("zabij");
      d.vz = v * v * o * o;
      d.va = v * o * o;
      d.vb = o * o;
      d.vi = o;
      d.vj = 1;
      timed_launch(kClsScatter, static_cast<double>(d.nzx) * o * o * v * v * 3 * sizeof(T), 0.0,
                   [&] { CU(launch_antisym4<T>(S2c, d, st())); });
    }
    amp_end();
  }

  bool is_fixed(const void* p) const {
    for (auto& kv : Vb)
      if (p >= kv.second.p && p < static_cast<const char*>(kv.second.p) + kv.second.bytes) return true;
    for (auto& kv : Fb)
      if (p >= kv.second.p && p < static_cast<const char*>(kv.second.p) + kv.second.bytes) return true;
    return false;
  }
  T* fixed_adjoint(const void* p) {
    for (auto* mp : {&Vb, &Fb})
      for (auto& kv : *mp)
        if (kv.second.p == p) {
          Buf& b = fixed_bar[p];
          if (!b.p) {
            ensure(h_, b, kv.second.bytes);
            CU(cudaMemsetAsync(b.p, 0, kv.second.bytes, st()));
          }
          return static_cast<T*>(b.p);
        }
    throw Fail{FTCC_ERR_STATE, "adjoint of an unknown fixed operand"};
  }
  void zero(T* p, const char* L) {
    long long n = 1;
    for (const char* q = L; *q; ++q) n *= dimof(*q);
    CU(cudaMemsetAsync(p, 0, n * sizeof(T), st()));
  }
  T* adj(const void* p) {
    auto it = bar.find(p);
    if (it == bar.end()) throw Fail{FTCC_ERR_STATE, "tape operand without adjoint"};
    return it->second;
  }

  // Vector-Jacobian product of the S kernel for nx tau slices of every
  // instance: given cotangents w1 (S1 shape) and w2 (S2 shape), overwrites
  // t1bar, t2bar with (dS/ds)^T w.  w1 and w2 are used as scratch.  With
  // want_fixed_bar the adjoints of the integral and Fock blocks accumulate in
  // fixed_bar (not cleared here).
  void vjp(const T* t1c, const T* t2c, T* w1, T* w2, T* t1bar, T* t2bar, int nxcur) {
    if (sp) {
      sparse_vjp(t1c, t2c, w1, w2, t1bar, t2bar, nxcur);
      return;
    }
    const long long o = no, v = nv, x = static_cast<long long>(nxcur) * nz;
    // adjoint buffers sized like the chunk intermediates
    Buf* pairs[][2] = {{&bta, &ta}, {&bX, &X}, {&bWmnij, &Wmnij}, {&bWabef, &Wabef}, {&bWmbej, &Wmbej},
                       {&bY, &Y}, {&bFae, &Fae}, {&bFmi, &Fmi}, {&bFme, &Fme}, {&bFt, &Ft}, {&bFt2, &Ft2},
                       {&bR, &R}, {&bR2, &R2}};
    for (auto& pr : pairs) {
      ensure(h_, *pr[0], pr[1]->bytes);
      CU(cudaMemsetAsync(pr[0]->p, 0, pr[1]->bytes, st()));
    }
    const size_t big = std::max(std::max(o * o * v * v, v * v * v * v), o * o * o * o) * static_cast<size_t>(x) * sizeof(T);
    ensure(h_, bD, big);
    ensure(h_, bP, x * o * o * v * v * sizeof(T));
    ensure(h_, bQ, x * o * o * v * v * sizeof(T));
    ensure(h_, sx1, x * o * v * sizeof(T));
    ensure(h_, sx2, x * o * o * v * v * sizeof(T));
    ensure(h_, ones, static_cast<size_t>(nz) * nxc * sizeof(T));
    {
      std::vector<T> h1(static_cast<size_t>(nz) * nxc, T(1));
      CU(cudaMemcpyAsync(ones.p, h1.data(), h1.size() * sizeof(T), cudaMemcpyHostToDevice, st()));
      CU(cudaStreamSynchronize(st()));
    }
    // forward pass on the tape
    tape.clear();
    recording = true;
    try {
      s_kernel(t1c, t2c, static_cast<T*>(sx1.p), static_cast<T*>(sx2.p), nxcur);
    } catch (...) {
      recording = false;
      throw;
    }
    recording = false;
    bar.clear();
    for (auto& pr : pairs) bar[pr[1]->p] = static_cast<T*>(pr[0]->p);
    bar[sx1.p] = w1;
    bar[sx2.p] = w2;
    bar[t1c] = t1bar;
    bar[t2c] = t2bar;
    CU(cudaMemsetAsync(t1bar, 0, x * o * v * sizeof(T), st()));
    CU(cudaMemsetAsync(t2bar, 0, x * o * o * v * v * sizeof(T), st()));
    using CT = Tn<const T>;
    T* dbuf = static_cast<T*>(bD.p);
    for (auto it = tape.rbegin(); it != tape.rend(); ++it) {
      const Op& op = *it;
      if (op.kind == 0) {
        T* cb = adj(op.C);
        const T* D = cb;
        if (op.alpha != 1.0 || !op.anti.empty()) {
          scatter(dbuf, op.Lc.c_str(), cb, op.Lc.c_str(), op.alpha, 0.0, op.anti.c_str());
          D = dbuf;
        }
        for (int side = 0; side < 2; ++side) {
          const T* X = side == 0 ? op.A : op.B;
          const std::string& LX = side == 0 ? op.La : op.Lb;
          const T* Y = side == 0 ? op.B : op.A;
          const std::string& LY = side == 0 ? op.Lb : op.La;
          T* xb = nullptr;
          if (!is_fixed(X)) xb = adj(X);
          else if (want_fixed_bar) xb = fixed_adjoint(X);
          if (xb) contract({xb, LX.c_str()}, 1.0, CT{D, op.Lc.c_str()}, CT{Y, LY.c_str()}, "", 1.0);
        }
        if (op.beta == 0.0) zero(cb, op.Lc.c_str());
      } else if (op.kind == 1) {
        T* db = adj(op.C);
        if (!is_fixed(op.A)) {
          scatter(adj(op.A), op.La.c_str(), db, op.Lc.c_str(), op.alpha, 1.0, op.anti.c_str());
        } else if (want_fixed_bar) {
          // broadcast copy of a block over tau: its adjoint sums over tau
          const T* src = db;
          if (!op.anti.empty()) {
            scatter(dbuf, op.Lc.c_str(), db, op.Lc.c_str(), 1.0, 0.0, op.anti.c_str());
            src = dbuf;
          }
          contract({fixed_adjoint(op.A), op.La.c_str()}, op.alpha, CT{src, op.Lc.c_str()}, CT{static_cast<const T*>(ones.p), "zx"}, "",
                   1.0);
        }
        if (op.beta == 0.0) zero(db, op.Lc.c_str());
      } else if (op.kind == 2) {
        // tt = t2 + 1/2 p (when built), ta = t2 + p, p_ijab = t_ia t_jb - t_ib t_ja
        T* ttb = op.C ? adj(op.C) : nullptr;
        T* tab = adj(op.C2);
        T* t2b = adj(op.B);
        T* t1b = adj(op.A);
        T* P = static_cast<T*>(bP.p);
        T* Q = static_cast<T*>(bQ.p);
        if (ttb) scatter(t2b, "zxijab", ttb, "zxijab", 1.0, 1.0, "");
        scatter(t2b, "zxijab", tab, "zxijab", 1.0, 1.0, "");
        scatter(P, "zxijab", tab, "zxijab", 1.0, 0.0, "");
        if (ttb) scatter(P, "zxijab", ttb, "zxijab", 0.5, 1.0, "");
        scatter(Q, "zxijab", P, "zxijab", 1.0, 0.0, "ijab");
        contract({t1b, "zxkc"}, 1.0, CT{Q, "zxkjcb"}, CT{op.A, "zxjb"}, "", 1.0);
      } else {
        // X[j,n,f,b] = 1/2 t2[j,n,f,b] + t1[j,f] t1[n,b]
        T* xb = adj(op.C);
        T* t2b = adj(op.B);
        T* t1b = adj(op.A);
        scatter(t2b, "zxjnfb", xb, "zxjnfb", 0.5, 1.0, "");
        contract({t1b, "zxjf"}, 1.0, CT{xb, "zxjnfb"}, CT{op.A, "zxnb"}, "", 1.0);
        contract({t1b, "zxnb"}, 1.0, CT{xb, "zxjnfb"}, CT{op.A, "zxjf"}, "", 1.0);
      }
    }
  }
};

Batch::~Batch() {
  s32.reset();
  s64.reset();
  for (Inst& I : inst) {
    Buf* bs[] = {&I.n, &I.nbar, &I.f, &I.fbar, &I.facO, &I.facV};
    for (Buf* q : bs) home->put(*q);
  }
  Buf* bs[] = {&idxO, &idxV, &em, &ep, &hz, &V64, &F64, &state, &live, &m1, &m2, &mn1, &mn2, &u1, &u2, &tb1,
               &tb2, &dE1, &cz, &lpart, &facOz, &facVz, &epsz};
  for (Buf* q : bs) home->put(*q);
}

SpTables::~SpTables() {
  Buf* bs[] = {&imp, &ssum.ent, &ssum.kl, &ssum.sec, &ssum.work, &sdiff.ent, &sdiff.kl, &sdiff.sec, &sdiff.work,
               &ssum_u.ent, &ssum_u.kl, &ssum_u.sec, &ssum_u.work, &ssum.work_small, &sdiff.work_small,
               &ssum_u.work_small, &canon, &vl1, &voff1, &vl2, &voff2, &vall, &vswap, &vrot};
  for (Buf* q : bs) home->put(*q);
}

// ---- block-sparse tables (host)
namespace {
std::array<int, 4> canon_charge(std::array<int, 4> q, const int* mod) {
  for (int k = 0; k < 4; ++k)
    if (mod[k] > 0) q[k] = ((q[k] % mod[k]) + mod[k]) % mod[k];
  return q;
}
uint64_t charge_key(const std::array<int, 4>& q) {
  uint64_t key = 0;
  for (int k = 0; k < 4; ++k) key = (key << 16) | static_cast<uint16_t>(q[k] + 32768);
  return key;
}
}  // namespace

// Pairs (p, q) of orbitals grouped by the charge q_p + q_q (diff = false) or
// q_p - q_q, in order of first appearance over p-major (p, q); within a
// sector the pairs are p-ascending and no two share p (nor q), since the
// orbitals' charges are distinct.
std::vector<std::vector<int2>> pair_sectors(const ftcc_ctx* c, int n, bool diff, bool unordered,
                                            std::vector<int>* sector_of = nullptr) {
  std::unordered_map<uint64_t, int> sid;
  std::vector<std::vector<int2>> rows;
  if (sector_of) sector_of->assign(static_cast<size_t>(n) * n, -1);
  for (int p = 0; p < n; ++p)
    for (int q = unordered ? p + 1 : 0; q < n; ++q) {
      std::array<int, 4> ch;
      for (int k = 0; k < 4; ++k) ch[k] = c->charge[p][k] + (diff ? -c->charge[q][k] : c->charge[q][k]);
      const uint64_t key = charge_key(canon_charge(ch, c->charge_mod));
      auto it = sid.find(key);
      if (it == sid.end()) {
        it = sid.emplace(key, static_cast<int>(rows.size())).first;
        rows.emplace_back();
      }
      rows[it->second].push_back(make_int2(p, q));
      if (sector_of) (*sector_of)[static_cast<size_t>(p) * n + q] = it->second;
    }
  return rows;
}

// imp[a][b][c] = the orbital d with q_d = q_a + q_b - q_c, or -1: (c, d) is
// then a pair of the sum sector of (a, b), so the table and every list of
// valid positions are read off the sectors without visiting a hole.
void build_implied(SpTables& B, const ftcc_ctx* c) {
  const int n = B.n;
  std::unordered_map<uint64_t, int> orb;
  for (int p = 0; p < n; ++p) orb[charge_key(canon_charge(c->charge[p], c->charge_mod))] = p;
  if (static_cast<int>(orb.size()) != n) throw Fail{FTCC_ERR_INVALID_ARG, "block_sparse: two orbitals share a charge"};
  std::vector<int> ssec, dsec;
  const std::vector<std::vector<int2>> srows = pair_sectors(c, n, false, false, &ssec);
  const std::vector<std::vector<int2>> drows = pair_sectors(c, n, true, false, &dsec);
  // second letters of every difference sector, ascending
  std::vector<std::vector<int>> dsecond(drows.size());
  for (size_t s = 0; s < drows.size(); ++s) {
    for (const int2& e : drows[s]) dsecond[s].push_back(e.y);
    std::sort(dsecond[s].begin(), dsecond[s].end());
  }
  const long long n3 = static_cast<long long>(n) * n * n;
  std::vector<int16_t> t(n3, -1);
  // valid positions (p0, p1, p2) ascending: p2 runs over the first letters of
  // the sum sector of (p0, p1), which are ascending
  std::vector<int> va, vs, vr, cp;
  std::vector<int> o1(n + 1, 0), o2(n + 1, 0);
  va.reserve(n3 / 4);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      const int base = (a * n + b) * n;
      int16_t* row = t.data() + base;
      const std::vector<int2>& sec = srows[ssec[static_cast<size_t>(a) * n + b]];
      o2[a + 1] += static_cast<int>(sec.size());
      for (const int2& e : sec) {
        row[e.x] = static_cast<int16_t>(e.y);
        va.push_back(base + e.x);
        ++o1[e.x + 1];
        // canonical positions of the antisymmetric doubles: a < b, p2 < implied
        if (a < b && e.x < e.y) cp.push_back(base + e.x);
      }
    }
  // (p0, p2, p1) valid: q_p0 - q_p1 = q_d - q_p2, p2 a second letter of the
  // difference sector of (p0, p1); (p1, p2, p0) valid: p2 a second letter of
  // the difference sector of (p1, p0)
  vs.reserve(va.size());
  vr.reserve(va.size());
  for (int p0 = 0; p0 < n; ++p0)
    for (int p1 = 0; p1 < n; ++p1) {
      const int base = (p0 * n + p1) * n;
      for (int p2 : dsecond[dsec[static_cast<size_t>(p0) * n + p1]]) vs.push_back(base + p2);
      for (int p2 : dsecond[dsec[static_cast<size_t>(p1) * n + p0]]) vr.push_back(base + p2);
    }
  // per orbital p, the valid positions (m, q, p) and (p, m, q) as m n + q,
  // ascending: (p, m, q) is a slice of the valid list, (m, q, p) a stable
  // bucketing of it by its last letter
  std::vector<int> l1(va.size()), l2(va.size());
  for (int p = 0; p < n; ++p) {
    o1[p + 1] += o1[p];
    o2[p + 1] += o2[p];
  }
  {
    std::vector<int> pos(o1.begin(), o1.end() - 1);
    size_t k = 0;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (const int2& e : srows[ssec[static_cast<size_t>(a) * n + b]]) {
          l1[pos[e.x]++] = a * n + b;
          l2[k++] = b * n + e.x;
        }
  }
  auto upload = [&](Buf& b, const std::vector<int>& v) {
    ensure(B.home, b, std::max<size_t>(1, v.size()) * sizeof(int));
    if (!v.empty()) CU(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, B.home->st));
  };
  ensure(B.home, B.imp, n3 * sizeof(int16_t));
  CU(cudaMemcpyAsync(B.imp.p, t.data(), n3 * sizeof(int16_t), cudaMemcpyHostToDevice, B.home->st));
  upload(B.vl1, l1);
  upload(B.voff1, o1);
  upload(B.vl2, l2);
  upload(B.voff2, o2);
  upload(B.vall, va);
  upload(B.vswap, vs);
  upload(B.vrot, vr);
  upload(B.canon, cp);
  B.nvall = static_cast<int>(va.size());
  B.nvswap = static_cast<int>(vs.size());
  B.nvrot = static_cast<int>(vr.size());
  B.ncanon = static_cast<long long>(cp.size());
  CU(cudaStreamSynchronize(B.home->st));
}

// sectors of ordered pairs (p, q) by q_p + q_q (diff = false) or q_p - q_q;
// the summed index of a sector runs over the first (sum) or second (diff)
// letters of its pairs
void build_sectors(SpTables& B, const ftcc_ctx* c, bool diff, SecTab& T, bool unordered = false) {
  const int n = B.n, tile = sector_tile();
  const std::vector<std::vector<int2>> rows = pair_sectors(c, n, diff, unordered);
  std::vector<int2> ent;
  std::vector<int> kl;
  std::vector<int4> sec, work, work_small;
  T.flops = 0;
  for (size_t s = 0; s < rows.size(); ++s) {
    const int off = static_cast<int>(ent.size()), cnt = static_cast<int>(rows[s].size());
    for (const int2& e : rows[s]) {
      ent.push_back(e);
      kl.push_back(diff ? e.y : e.x);
    }
    sec.push_back(make_int4(off, cnt, off, cnt));
    if (cnt <= 16) {
      work_small.push_back(make_int4(static_cast<int>(s), 0, 0, 0));
    } else {
      for (int r0 = 0; r0 < cnt; r0 += tile)
        for (int c0 = 0; c0 < cnt; c0 += tile) work.push_back(make_int4(static_cast<int>(s), r0, c0, 0));
    }
    T.flops += 2.0 * cnt * static_cast<double>(cnt) * cnt;
  }
  ftcc_ctx* h = B.home;
  ensure(h, T.ent, ent.size() * sizeof(int2));
  ensure(h, T.kl, kl.size() * sizeof(int));
  ensure(h, T.sec, sec.size() * sizeof(int4));
  ensure(h, T.work, std::max<size_t>(1, work.size()) * sizeof(int4));
  ensure(h, T.work_small, std::max<size_t>(1, work_small.size()) * sizeof(int4));
  if (!work_small.empty())
    CU(cudaMemcpyAsync(T.work_small.p, work_small.data(), work_small.size() * sizeof(int4), cudaMemcpyHostToDevice,
                       h->st));
  CU(cudaMemcpyAsync(T.ent.p, ent.data(), ent.size() * sizeof(int2), cudaMemcpyHostToDevice, h->st));
  CU(cudaMemcpyAsync(T.kl.p, kl.data(), kl.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CU(cudaMemcpyAsync(T.sec.p, sec.data(), sec.size() * sizeof(int4), cudaMemcpyHostToDevice, h->st));
  if (!work.empty())
    CU(cudaMemcpyAsync(T.work.p, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice, h->st));
  CU(cudaStreamSynchronize(h->st));
  T.nwork = static_cast<int>(work.size());
  T.nwork_small = static_cast<int>(work_small.size());
}

}  // namespace ftcc

using namespace ftcc;

namespace {

const char* kStatusText[] = {"ok", "invalid argument", "no CUDA device", "out of device memory", "not converged",
                             "diverged", "device wait timed out", "unsupported", "call order violated",
                             "CUDA error"};

ftcc_options default_options() {
  ftcc_options o;
  o.tol_omega = 1e-10;
  o.tol_amp = 1e-8;
  o.damping = 1.0;
  o.trunc_thr = 0.0;
  o.max_iter = 200;
  o.precision = FTCC_PREC_FP64;
  o.refine_max_iter = 2;
  o.tol_mixed = 1e-7;
  o.polish_max_iter = 40;
  o.fp64_propagation = 1;
  o.tol_refine = 1e-6;
  o.mixed_adjoint = 0;
  o.block_sparse = 0;
  o.tau_chunk = 0;
  o.use_graph = 1;
  o.stream_tau = 0;
  o.autotune = 1;
  return o;
}

void sync(ftcc_ctx* c) { CU(cudaStreamSynchronize(c->st)); }

void check_device_error(ftcc_ctx* c) {
  int e = 0;
  CU(cudaMemcpyAsync(&e, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  sync(c);
  if (e != 0) {
    CU(cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->st));
    throw Fail{FTCC_ERR_TIMEOUT, "a bounded device wait expired (code " + std::to_string(e) + ")"};
  }
}

// Thermal integral and Fock blocks of every instance, stacked [z][block].
template <class T>
void build_blocks(Batch& B, Solver<T>& s) {
  ftcc_ctx* h = B.home;
  const int o = B.no, v = B.nv;
  const char* eri_pat[] = {"oovv", "ovvv", "ooov", "oooo", "vvvv", "vovv", "ovvo", "oovo", "ovov", "vvoo", "vvvo", "ovoo"};
  for (const char* pat : eri_pat) {
    int nn[4];
    long long total = 1;
    for (int k = 0; k < 4; ++k) {
      nn[k] = pat[k] == 'o' ? o : v;
      total *= nn[k];
    }
    Buf& buf = s.Vb[pat];
    ensure(h, buf, total * B.nz * sizeof(T));
    for (int z = 0; z < B.nz; ++z) {
      const Inst& I = B.inst[z];
      const int* ix[4];
      const double* fx[4];
      for (int k = 0; k < 4; ++k) {
        const bool ho = pat[k] == 'o';
        ix[k] = static_cast<const int*>(ho ? B.idxO.p : B.idxV.p);
        fx[k] = static_cast<const double*>(ho ? I.facO.p : I.facV.p);
      }
      CU(launch_thermal_eri<T>(static_cast<const double*>(I.ctx->eri.p), B.N, ix[0], fx[0], nn[0], ix[1], fx[1], nn[1],
                               ix[2], fx[2], nn[2], ix[3], fx[3], nn[3], static_cast<T*>(buf.p) + z * total, h->st));
    }
  }
  const char* f_pat[] = {"ov", "vv", "oo", "vo"};
  for (const char* pat : f_pat) {
    const bool h0 = pat[0] == 'o', h1 = pat[1] == 'o';
    const long long total = static_cast<long long>(h0 ? o : v) * (h1 ? o : v);
    Buf& buf = s.Fb[pat];
    ensure(h, buf, total * B.nz * sizeof(T));
    for (int z = 0; z < B.nz; ++z) {
      const Inst& I = B.inst[z];
      CU(launch_thermal_fock<T>(static_cast<const double*>(I.fbar.p), B.N,
                                static_cast<const int*>(h0 ? B.idxO.p : B.idxV.p),
                                static_cast<const double*>(h0 ? I.facO.p : I.facV.p), h0 ? o : v,
                                static_cast<const int*>(h1 ? B.idxO.p : B.idxV.p),
                                static_cast<const double*>(h1 ? I.facO.p : I.facV.p), h1 ? o : v,
                                static_cast<T*>(buf.p) + z * total, h->st));
    }
  }
}

// The thermal integral and Fock blocks in block-sparse storage: each ERI
// class as an N^3 array (fourth index implied), each Fock class as its
// diagonal.  No truncation, so the hole and particle lists are every orbital.
template <class T>
void build_blocks_sparse(Batch& B, Solver<T>& s) {
  ftcc_ctx* h = B.home;
  const int n = B.N;
  const long long n3 = static_cast<long long>(n) * n * n;
  const Inst& I = B.inst[0];
  const int16_t* imp = static_cast<const int16_t*>(B.imp.p);
  auto fac = [&](char c) { return static_cast<const double*>(c == 'o' ? I.facO.p : I.facV.p); };
  const char* eri_pat[] = {"oovv", "ovvv", "ooov", "oooo", "vvvv", "vovv", "ovvo", "oovo", "ovov", "vvoo", "vvvo", "ovoo"};
  for (const char* pat : eri_pat) {
    Buf& buf = s.Vb[pat];
    ensure(h, buf, n3 * sizeof(T));
    CU(launch_sp_thermal_eri<T>(static_cast<const double*>(I.ctx->eri.p), imp, n, fac(pat[0]), fac(pat[1]),
                                fac(pat[2]), fac(pat[3]), static_cast<T*>(buf.p), h->st));
  }
  const char* f_pat[] = {"ov", "vv", "oo", "vo"};
  for (const char* pat : f_pat) {
    Buf& buf = s.Fb[pat];
    ensure(h, buf, n * sizeof(T));
    CU(launch_sp_thermal_fock<T>(static_cast<const double*>(I.fbar.p), n, fac(pat[0]), fac(pat[1]),
                                 static_cast<T*>(buf.p), h->st));
  }
}

template <class T>
Solver<T>& make_solver(Batch& B, int kind) {
  std::unique_ptr<Solver<T>>* slot;
  if constexpr (sizeof(T) == 8) slot = &B.s64;
  else slot = &B.s32;
  if (!*slot || (*slot)->gk != kind) {
    slot->reset(new Solver<T>(&B, kind));
    Solver<T>& s = **slot;
    ftcc_ctx* h = B.home;
    s.nz = B.nz;
    s.no = B.no;
    s.nv = B.nv;
    s.ng = B.ng;
    {
      if (B.sparse) {
        s.sp = true;
        s.nxc = B.opt.tau_chunk > 0 ? std::min(B.opt.tau_chunk, B.ng) : B.ng;
        build_blocks_sparse(B, s);
        const long long g = s.ng, n1 = s.n1(), n2 = s.n2();
        ensure(h, s.t1, g * n1 * sizeof(T));
        ensure(h, s.t2, g * n2 * sizeof(T));
        ensure(h, s.S1, g * n1 * sizeof(T));
        ensure(h, s.S2, g * n2 * sizeof(T));
        CU(cudaMemsetAsync(s.t1.p, 0, g * n1 * sizeof(T), h->st));
        CU(cudaMemsetAsync(s.t2.p, 0, g * n2 * sizeof(T), h->st));
        // S2 is written through its canonical elements only: the elements with
        // i = j or a = b stay zero
        CU(cudaMemsetAsync(s.S2.p, 0, g * n2 * sizeof(T), h->st));
        s.sparse_alloc();
        s.nb1 = std::max(1, std::min(prop_blocks() + 1, static_cast<int>((n1 + 127) / 128)));
        s.nb2 = std::max(1, std::min(prop_blocks() + 1, static_cast<int>((B.ncanon + 127) / 128)));
        ensure(h, s.part1, static_cast<size_t>(s.nb1) * (s.ng + 2) * sizeof(double));
        ensure(h, s.part2, static_cast<size_t>(s.nb2) * (s.ng + 2) * sizeof(double));
        return s;
      }
    }
    s.stream = B.nz == 1 && B.opt.stream_tau != 0;
    if (s.stream) s.nxc = std::min(B.ng, B.opt.tau_chunk > 0 ? B.opt.tau_chunk : 1);
    else s.nxc = (B.nz == 1 && B.opt.tau_chunk > 0) ? std::min(B.opt.tau_chunk, B.ng) : B.ng;
    build_blocks<T>(B, s);
    const long long o = s.no, v = s.nv, g = static_cast<long long>(s.ng) * s.nz;
    // tau slices of S kept: all of them, or (streamed) one propagation window
    // of max(3, tau_chunk) points
    const long long gS = s.stream ? std::min(s.ng, std::max(3, s.nxc)) : g;
    ensure(h, s.t1, g * o * v * sizeof(T));
    ensure(h, s.t2, g * o * o * v * v * sizeof(T));
    ensure(h, s.S1, gS * o * v * sizeof(T));
    ensure(h, s.S2, gS * o * o * v * v * sizeof(T));
    if (s.stream) {
      ensure(h, s.ch1, 5 * o * v * sizeof(T));
      ensure(h, s.ch2, 5 * o * o * v * v * sizeof(T));
    }
    CU(cudaMemsetAsync(s.t1.p, 0, g * o * v * sizeof(T), h->st));
    CU(cudaMemsetAsync(s.t2.p, 0, g * o * o * v * v * sizeof(T), h->st));
    s.alloc_chunk();
    s.nb1 = std::max(1, std::min(prop_blocks() / s.nz + 1, static_cast<int>((o * v + 127) / 128)));
    s.nb2 = std::max(1, std::min(prop_blocks() / s.nz + 1, static_cast<int>((o * o * v * v + 127) / 128)));
    ensure(h, s.part1, static_cast<size_t>(s.nz) * s.nb1 * (s.ng + 2) * sizeof(double));
    ensure(h, s.part2, static_cast<size_t>(s.nz) * s.nb2 * (s.ng + 2) * sizeof(double));
  }
  return **slot;
}

PropArgs prop_args(Batch& B, int nslot) {
  PropArgs a{};
  a.ng = B.ng;
  a.no = B.no;
  a.nv = B.nv;
  a.nz = B.nz;
  a.N = B.N;
  a.idxO = static_cast<const int*>(B.idxO.p);
  a.idxV = static_cast<const int*>(B.idxV.p);
  a.em = static_cast<const double*>(B.em.p);
  a.ep = static_cast<const double*>(B.ep.p);
  a.hz = static_cast<const double*>(B.hz.p);
  a.live = static_cast<const int*>(B.live.p);
  a.damping = B.opt.damping;
  a.nslot = nslot;
  a.size = nslot == 2 ? static_cast<long long>(B.no) * B.nv : static_cast<long long>(B.no) * B.no * B.nv * B.nv;
  if (B.sparse) {
    a.size = nslot == 2 ? B.N : static_cast<long long>(B.N) * B.N * B.N;
    a.imp = static_cast<const int16_t*>(B.imp.p);
    if (nslot == 4) {
      a.canon = static_cast<const int*>(B.canon.p);
      a.ncanon = B.ncanon;
    }
  }
  a.y0 = 0;
  a.y1 = B.ng;
  a.s_ng = B.ng;
  a.chain = nullptr;
  return a;
}

// Arithmetic of the propagation in an FP32 sweep (option fp64_propagation):
// the element ratios exp(-Delta h) always come from the FP64 tables; the
// recurrence and the energy sums run in FP64 (2), the sums only (1) or
// neither (0).
template <class T>
void set_tables(Batch& B, PropArgs& a) {
  if (sizeof(T) == 4) a.arith64 = B.opt.fp64_propagation;
}

// One application of the fixed-point map to every tau point of every instance.
template <class T>
void iterate_once(Batch& B, Solver<T>& s) {
  s.prof_next = 0;
  const long long n1 = s.n1(), n2 = s.n2();
  if (s.stream) {
    // S for one chunk of tau points at a time, then the propagation of those
    // points from the carried chain state (the S kernel at tau_x reads only
    // the amplitudes at tau_x, which the propagation of earlier chunks left
    // untouched; the first chunk has at least three points)
    for (int x0 = 0; x0 < s.ng;) {
      // propagation window: the first one spans at least three points (S_2
      // enters the y = 1 step); the S kernel runs tau_chunk points at a time
      const int nx = std::min(x0 == 0 ? std::max(3, s.nxc) : s.nxc, s.ng - x0);
      for (int xs = 0; xs < nx; xs += s.nxc) {
        const int nk = std::min(s.nxc, nx - xs);
        s.s_kernel(static_cast<T*>(s.t1.p) + (x0 + xs) * n1, static_cast<T*>(s.t2.p) + (x0 + xs) * n2,
                   static_cast<T*>(s.S1.p) + xs * n1, static_cast<T*>(s.S2.p) + xs * n2, nk);
      }
      for (int pass = 0; pass < 2; ++pass) {
        PropArgs a = prop_args(B, pass == 0 ? 2 : 4);
        set_tables<T>(B, a);
        a.wE = static_cast<const double*>(pass == 0 ? B.F64.p : B.V64.p);
        a.cE = pass == 0 ? 1.0 : 0.25;
        a.t1E = pass == 0 ? nullptr : s.t1.p;
        a.partials = static_cast<double*>(pass == 0 ? s.part1.p : s.part2.p);
        a.nblocks = pass == 0 ? s.nb1 : s.nb2;
        a.y0 = x0;
        a.y1 = x0 + nx;
        a.s_ng = nx;
        a.chain = pass == 0 ? s.ch1.p : s.ch2.p;
        const long long n = pass == 0 ? n1 : n2;
        const double bytes = static_cast<double>(nx) * n * 3 * sizeof(T) + static_cast<double>(n) * (8 + 10 * sizeof(T));
        s.timed_launch(kClsPropagate, bytes, 0.0, [&] {
          CU(launch_propagate<T>(static_cast<const T*>(pass == 0 ? s.S1.p : s.S2.p),
                                 static_cast<T*>(pass == 0 ? s.t1.p : s.t2.p), a, B.home->st));
        });
      }
      x0 += nx;
    }
    CU(launch_reduce(static_cast<const double*>(s.part1.p), s.nb1, static_cast<const double*>(s.part2.p), s.nb2,
                     s.ng, B.nz, static_cast<const double*>(B.hz.p), static_cast<const int*>(B.live.p),
                     static_cast<double*>(B.state.p), B.home->st));
    return;
  }
  for (int x0 = 0; x0 < s.ng; x0 += s.nxc) {   // tau chunks only when nz == 1
    const int nx = std::min(s.nxc, s.ng - x0);
    s.s_kernel(static_cast<T*>(s.t1.p) + x0 * n1, static_cast<T*>(s.t2.p) + x0 * n2, static_cast<T*>(s.S1.p) + x0 * n1,
               static_cast<T*>(s.S2.p) + x0 * n2, nx);
  }
  PropArgs a = prop_args(B, 2);
  set_tables<T>(B, a);
  a.wE = static_cast<const double*>(B.F64.p);
  a.cE = 1.0;
  a.t1E = nullptr;
  a.partials = static_cast<double*>(s.part1.p);
  a.nblocks = s.nb1;
  const double b1 = static_cast<double>(B.nz) * s.ng * n1 * 3 * sizeof(T) + static_cast<double>(B.nz) * n1 * 8;
  s.timed_launch(kClsPropagate, b1, 0.0,
                 [&] { CU(launch_propagate<T>(static_cast<const T*>(s.S1.p), static_cast<T*>(s.t1.p), a, B.home->st)); });
  a = prop_args(B, 4);
  set_tables<T>(B, a);
  a.wE = static_cast<const double*>(B.V64.p);
  a.cE = 0.25;
  a.t1E = s.t1.p;
  a.partials = static_cast<double*>(s.part2.p);
  a.nblocks = s.nb2;
  const double b2 = static_cast<double>(B.nz) * s.ng * n2 * 3 * sizeof(T) + static_cast<double>(B.nz) * n2 * 8;
  s.timed_launch(kClsPropagate, b2, 0.0,
                 [&] { CU(launch_propagate<T>(static_cast<const T*>(s.S2.p), static_cast<T*>(s.t2.p), a, B.home->st)); });
  CU(launch_reduce(static_cast<const double*>(s.part1.p), s.nb1, static_cast<const double*>(s.part2.p), s.nb2, s.ng,
                   B.nz, static_cast<const double*>(B.hz.p), static_cast<const int*>(B.live.p),
                   static_cast<double*>(B.state.p), B.home->st));
}

template <class T>
void run_iterations(Batch& B, Solver<T>& s, int n) {
  ftcc_ctx* h = B.home;
  for (int k = 0; k < n; ++k) {
    if (B.opt.use_graph && s.gexec) {
      CU(cudaGraphLaunch(s.gexec, h->st));
    } else if (B.opt.use_graph && s.warm) {
      // capture after one uncaptured iteration has sized every workspace
      cudaGraph_t g;
      CU(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
      try {
        iterate_once<T>(B, s);
      } catch (...) {
        cudaStreamEndCapture(h->st, &g);
        throw;
      }
      CU(cudaStreamEndCapture(h->st, &g));
      size_t nn = 0;
      CU(cudaGraphGetNodes(g, nullptr, &nn));
      s.graph_nodes = static_cast<int>(nn);
      CU(cudaGraphInstantiate(&s.gexec, g, 0));
      if (s.graph) cudaGraphDestroy(s.graph);
      s.graph = g;   // kept: a batched step embeds it in one graph with the other batches'
      ++s.graph_gen;
      CU(cudaGraphLaunch(s.gexec, h->st));
    } else {
      iterate_once<T>(B, s);
      s.warm = true;
    }
  }
}

template <class T>
void collect_profile(Batch& B, Solver<T>& s) {
  if (!s.profiling || s.prof_next == 0) return;
  CU(cudaStreamSynchronize(B.home->st));
  for (size_t i = 0; i < s.prof_next; ++i) {
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, s.prof[i].e0, s.prof[i].e1));
    const int c = s.prof[i].cls;
    B.prof_ms[c] += ms;
    B.prof_bytes[c] += s.prof[i].bytes;
    B.prof_flops[c] += s.prof[i].flops;
    B.prof_launches[c] += 1;
  }
}

void run_batch(Batch& B, int n) {
  // with kernel timing on, each iteration is replayed and read back on its own
  const bool prof = B.active == 1 ? (B.s32 && B.s32->profiling) : (B.s64 && B.s64->profiling);
  const int reps = prof ? n : 1, per = prof ? 1 : n;
  for (int r = 0; r < reps; ++r) {
    if (B.active == 1) {
      run_iterations<float>(B, *B.s32, per);
      collect_profile<float>(B, *B.s32);
    } else {
      run_iterations<double>(B, *B.s64, per);
      collect_profile<double>(B, *B.s64);
    }
  }
  B.iterations += n;
}

void timed_iterations(Batch& B, int n) {
  ftcc_ctx* h = B.home;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, h->st));
  run_batch(B, n);
  CU(cudaEventRecord(e1, h->st));
  CU(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B.ms_total += ms;
  B.ms_count += n;
}

// state rows [z][kStateStride]: 0 Omega_CC, 1 |dOmega_CC|, 2 max|ds|/max(1,max|s|)
std::vector<double> read_states(Batch& B) {
  std::vector<double> s(static_cast<size_t>(B.nz) * kStateStride);
  CU(cudaMemcpyAsync(s.data(), B.state.p, s.size() * sizeof(double), cudaMemcpyDeviceToHost, B.home->st));
  sync(B.home);
  return s;
}

int kernels_per_iter(Batch& B) {
  if (B.active == 1) return B.s32 ? B.s32->graph_nodes : 0;
  return B.s64 ? B.s64->graph_nodes : 0;
}

void fill_result(Batch& B, int z, const std::vector<double>& st, ftcc_result* out) {
  if (!out) return;
  const Inst& I = B.inst[z];
  const double* s = st.data() + static_cast<size_t>(z) * kStateStride;
  out->omega0 = I.omega0;
  out->omega1 = I.omega1;
  out->omega_cc = s[0];
  out->omega = I.omega0 + I.omega1 + s[0];
  out->d_omega = s[1];
  out->d_amp = s[2];
  out->iterations = I.conv_iter > 0 ? I.conv_iter : B.iterations;
  out->refine_iterations = B.refine_iterations;
  out->polish_iterations = B.polish_iterations;
  out->converged = (B.live_host.empty() || B.live_host[z]) && (B.solved || I.conv_iter > 0) ? 1 : 0;
  out->n_occ = B.no;
  out->n_vir = B.nv;
  out->ms_per_iter = B.ms_count ? B.ms_total / B.ms_count : 0.0;
  out->kernels_per_iter = kernels_per_iter(B);
}

// Copy the FP32 amplitudes into the FP64 solver (refinement hand-over).
void promote_to_fp64(Batch& B) {
  Solver<double>& d = make_solver<double>(B, GEMM_F64);
  Solver<float>& s = *B.s32;
  const long long n1 = static_cast<long long>(s.nz) * s.ng * s.n1();
  const long long n2 = static_cast<long long>(s.nz) * s.ng * s.n2();
  CU(launch_convert<float, double>(static_cast<const float*>(s.t1.p), static_cast<double*>(d.t1.p), n1, B.home->st));
  CU(launch_convert<float, double>(static_cast<const float*>(s.t2.p), static_cast<double*>(d.t2.p), n2, B.home->st));
  B.active = 0;
}

ftcc_status run_guarded(ftcc_ctx* c, const std::function<ftcc_status()>& fn) {
  try {
    return fn();
  } catch (const Fail& f) {
    if (c) c->err = f.msg;
    return f.s;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "host allocation failed";
    return FTCC_ERR_OOM;
  }
}

void detach(ftcc_ctx* c) {
  if (!c->batch) return;
  std::shared_ptr<Batch> b = c->batch;
  c->batch.reset();
  // the batch lives while any member holds it; its memory belongs to home
  (void)b;
}

bool shell_grid(int n_pw, std::vector<int>& out) {
  int r = 0;
  while ((r + 1) * (r + 1) <= n_pw) ++r;
  r += 2;
  struct P { int n2, x, y, z; };
  std::vector<P> pts;
  for (int x = -r; x <= r; ++x)
    for (int y = -r; y <= r; ++y)
      for (int z = -r; z <= r; ++z) pts.push_back({x * x + y * y + z * z, x, y, z});
  std::sort(pts.begin(), pts.end(), [](const P& a, const P& b) {
    if (a.n2 != b.n2) return a.n2 < b.n2;
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
  });
  for (int cut = 0; cut <= 3 * r * r; ++cut) {
    int cnt = 0;
    for (const P& p : pts) cnt += p.n2 <= cut;
    if (cnt == n_pw) {
      out.clear();
      for (const P& p : pts)
        if (p.n2 <= cut) {
          out.push_back(p.x);
          out.push_back(p.y);
          out.push_back(p.z);
        }
      return true;
    }
    if (cnt > n_pw) return false;
  }
  return false;
}

ftcc_status check_options(ftcc_ctx* c, const ftcc_options& o) {
  if (!(o.damping > 0 && o.damping <= 1) || o.max_iter < 0 || o.refine_max_iter < 0 || o.polish_max_iter < 0 || o.trunc_thr < 0 ||
      o.fp64_propagation < 0 || o.fp64_propagation > 2 || !(o.tol_refine >= 0) || o.mixed_adjoint < 0 ||
      o.mixed_adjoint > 1 || o.block_sparse < 0 || o.block_sparse > 1 ||
      o.trunc_thr >= 0.5 || o.precision < 0 || o.precision > 2 || o.tau_chunk < 0 || o.stream_tau < 0 ||
      o.stream_tau > 1 || o.autotune < 0 || o.autotune > 1 || !(o.tol_omega >= 0) ||
      !(o.tol_amp >= 0) || !(o.tol_mixed >= 0))
    return fail(c, FTCC_ERR_INVALID_ARG, "options out of range");
  return FTCC_OK;
}

// Set up a batch of instances (reference quantities, truncation, Fermi-scaled
// blocks, propagator tables, s = 0).  Every member must have the same number
// of spin orbitals and, after truncation, the same hole / particle sets.
std::shared_ptr<Batch> prepare_batch(ftcc_ctx* const* cs, int n, const double* beta, const double* mu, int ngrid,
                                     const ftcc_options& o) {
  ftcc_ctx* home = cs[0];
  CU(cudaSetDevice(home->device));
  auto B = std::make_shared<Batch>();
  B->home = home;
  B->nz = n;
  B->N = home->N;
  B->ng = ngrid;
  B->opt = o;
  B->prec = o.precision;
  const int N = B->N;
  B->inst.resize(n);
  std::vector<char> keepO(N, 1), keepV(N, 1);
  std::vector<std::vector<char>> kO(n), kV(n);
  for (int z = 0; z < n; ++z) {
    Inst& I = B->inst[z];
    I.ctx = cs[z];
    I.beta = beta[z];
    I.mu = mu[z];
    I.hstep = beta[z] / (ngrid - 1);
    ensure(home, I.n, N * sizeof(double));
    ensure(home, I.nbar, N * sizeof(double));
    ensure(home, I.f, static_cast<size_t>(N) * N * sizeof(double));
    ensure(home, I.fbar, static_cast<size_t>(N) * N * sizeof(double));
    Buf scal = home->get(8 * sizeof(double));
    if (!scal.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
    CU(launch_reference(static_cast<const double*>(cs[z]->h.p), static_cast<const double*>(cs[z]->eri.p),
                        static_cast<const double*>(cs[z]->eps.p), N, I.beta, I.mu, static_cast<double*>(I.n.p),
                        static_cast<double*>(I.nbar.p), static_cast<double*>(I.f.p), static_cast<double*>(I.fbar.p),
                        static_cast<double*>(scal.p), home->st));
    I.n_host.assign(N, 0.0);
    I.nbar_host.assign(N, 0.0);
    double sc[3];
    CU(cudaMemcpyAsync(I.n_host.data(), I.n.p, N * sizeof(double), cudaMemcpyDeviceToHost, home->st));
    CU(cudaMemcpyAsync(I.nbar_host.data(), I.nbar.p, N * sizeof(double), cudaMemcpyDeviceToHost, home->st));
    CU(cudaMemcpyAsync(sc, scal.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, home->st));
    sync(home);
    home->put(scal);
    I.omega0 = sc[0];
    I.omega1 = sc[1];
    for (int p = 0; p < N; ++p) {
      const char ko = I.n_host[p] >= o.trunc_thr, kv = I.nbar_host[p] >= o.trunc_thr;
      if (z == 0) {
        keepO[p] = ko;
        keepV[p] = kv;
      } else if (ko != keepO[p] || kv != keepV[p]) {
        throw Fail{FTCC_ERR_INVALID_ARG, "batched instances need identical truncation sets"};
      }
    }
  }
  for (int p = 0; p < N; ++p) {
    if (keepO[p]) B->O.push_back(p);
    if (keepV[p]) B->V.push_back(p);
  }
  if (B->O.empty() || B->V.empty()) throw Fail{FTCC_ERR_INVALID_ARG, "truncation left an empty space"};
  B->no = static_cast<int>(B->O.size());
  B->nv = static_cast<int>(B->V.size());
  if (o.block_sparse) {
    if (n != 1) throw Fail{FTCC_ERR_INVALID_ARG, "block_sparse: one instance per solve"};
    if (static_cast<int>(home->charge.size()) != N)
      throw Fail{FTCC_ERR_INVALID_ARG, "block_sparse: the system has no conserved orbital charges (UEG or k-space Hubbard)"};
    if (B->no != N || B->nv != N) throw Fail{FTCC_ERR_INVALID_ARG, "block_sparse: truncation must keep every orbital"};
    if (static_cast<long long>(N) * N * N >= (1LL << 31))
      throw Fail{FTCC_ERR_INVALID_ARG, "block_sparse: N^3 positions must fit 32-bit indices (N <= 1290)"};
    B->sparse = true;
    if (!home->sptab || home->sptab->n != N) {
      home->sptab.reset();
      auto T = std::make_shared<SpTables>();
      T->home = home;
      T->n = N;
      build_implied(*T, home);
      build_sectors(*T, home, false, T->ssum);
      build_sectors(*T, home, true, T->sdiff);
      build_sectors(*T, home, false, T->ssum_u, true);
      home->sptab = T;
    }
    B->sp_owner = home->sptab;
    static_cast<SpTableView&>(*B) = *home->sptab;
  }
  ensure(home, B->idxO, B->O.size() * sizeof(int));
  ensure(home, B->idxV, B->V.size() * sizeof(int));
  CU(cudaMemcpyAsync(B->idxO.p, B->O.data(), B->O.size() * sizeof(int), cudaMemcpyHostToDevice, home->st));
  CU(cudaMemcpyAsync(B->idxV.p, B->V.data(), B->V.size() * sizeof(int), cudaMemcpyHostToDevice, home->st));
  ensure(home, B->em, static_cast<size_t>(n) * N * sizeof(double));
  ensure(home, B->ep, static_cast<size_t>(n) * N * sizeof(double));
  ensure(home, B->hz, static_cast<size_t>(n) * 2 * sizeof(double));
  const long long no = B->no, nv = B->nv;
  // energy weights <ij||ab> and f_ia (Eq. E) in the storage of the amplitudes
  const long long w2 = B->sparse ? static_cast<long long>(N) * N * N : no * no * nv * nv;
  const long long w1 = B->sparse ? N : no * nv;
  ensure(home, B->V64, static_cast<size_t>(n) * w2 * sizeof(double));
  ensure(home, B->F64, static_cast<size_t>(n) * w1 * sizeof(double));
  ensure(home, B->state, static_cast<size_t>(n) * kStateStride * sizeof(double));
  std::vector<double> hb(2 * n);
  for (int z = 0; z < n; ++z) {
    Inst& I = B->inst[z];
    std::vector<double> fo, fv;
    for (int p : B->O) fo.push_back(std::sqrt(I.n_host[p]));
    for (int p : B->V) fv.push_back(std::sqrt(I.nbar_host[p]));
    ensure(home, I.facO, fo.size() * sizeof(double));
    ensure(home, I.facV, fv.size() * sizeof(double));
    CU(cudaMemcpyAsync(I.facO.p, fo.data(), fo.size() * sizeof(double), cudaMemcpyHostToDevice, home->st));
    CU(cudaMemcpyAsync(I.facV.p, fv.data(), fv.size() * sizeof(double), cudaMemcpyHostToDevice, home->st));
    CU(launch_prop_tables(static_cast<const double*>(cs[z]->eps.p), N, I.hstep, static_cast<double*>(B->em.p) + z * N,
                          static_cast<double*>(B->ep.p) + z * N, home->st));
    const int* iO = static_cast<const int*>(B->idxO.p);
    const int* iV = static_cast<const int*>(B->idxV.p);
    const double* fO = static_cast<const double*>(I.facO.p);
    const double* fV = static_cast<const double*>(I.facV.p);
    if (B->sparse) {
      CU(launch_sp_thermal_eri(static_cast<const double*>(cs[z]->eri.p), static_cast<const int16_t*>(B->imp.p), N, fO,
                               fO, fV, fV, static_cast<double*>(B->V64.p), home->st));
      CU(launch_sp_thermal_fock(static_cast<const double*>(I.fbar.p), N, fO, fV, static_cast<double*>(B->F64.p),
                                home->st));
    } else {
      CU(launch_thermal_eri<double>(static_cast<const double*>(cs[z]->eri.p), N, iO, fO, B->no, iO, fO, B->no, iV, fV,
                                    B->nv, iV, fV, B->nv, static_cast<double*>(B->V64.p) + z * no * no * nv * nv,
                                    home->st));
      CU(launch_thermal_fock<double>(static_cast<const double*>(I.fbar.p), N, iO, fO, B->no, iV, fV, B->nv,
                                     static_cast<double*>(B->F64.p) + z * no * nv, home->st));
    }
    hb[z] = I.hstep;
    hb[n + z] = I.beta;
    if (z == 0) {
      ensure(home, B->facOz, static_cast<size_t>(n) * no * sizeof(double));
      ensure(home, B->facVz, static_cast<size_t>(n) * nv * sizeof(double));
      ensure(home, B->epsz, static_cast<size_t>(n) * N * sizeof(double));
    }
    CU(cudaMemcpyAsync(static_cast<double*>(B->facOz.p) + z * no, fo.data(), no * sizeof(double), cudaMemcpyHostToDevice,
                       home->st));
    CU(cudaMemcpyAsync(static_cast<double*>(B->facVz.p) + z * nv, fv.data(), nv * sizeof(double), cudaMemcpyHostToDevice,
                       home->st));
    CU(cudaMemcpyAsync(static_cast<double*>(B->epsz.p) + z * N, cs[z]->eps.p, N * sizeof(double), cudaMemcpyDeviceToDevice,
                       home->st));
    sync(home);   // the host vectors fo / fv must outlive their copies
  }
  CU(cudaMemcpyAsync(B->hz.p, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice, home->st));
  B->live_host.assign(n, 1);
  ensure(home, B->live, static_cast<size_t>(n) * sizeof(int));
  CU(cudaMemcpyAsync(B->live.p, B->live_host.data(), n * sizeof(int), cudaMemcpyHostToDevice, home->st));
  CU(cudaMemsetAsync(B->state.p, 0, static_cast<size_t>(n) * kStateStride * sizeof(double), home->st));
  if (B->prec == FTCC_PREC_FP64) {
    make_solver<double>(*B, GEMM_F64);
    B->active = 0;
  } else if (B->sparse) {
    // FP32 storage and arithmetic on the SIMT pipes (the sector products are
    // small dense blocks); no tensor-core phases, so no polishing phase
    make_solver<float>(*B, GEMM_BF16X3);
    B->active = 1;
  } else {
    if (!tma_available()) throw Fail{FTCC_ERR_UNSUPPORTED, "tensor-map encoder unavailable in the driver"};
    make_solver<float>(*B, B->prec == FTCC_PREC_TF32 ? GEMM_TF32 : GEMM_BF16X3);
    B->active = 1;
  }
  sync(home);
  for (int z = 0; z < n; ++z) {
    detach(cs[z]);
    cs[z]->batch = B;
    cs[z]->member = z;
  }
  return B;
}

// Fixed-point loop of a prepared batch (see ft_ccsd_solve).
// Alg. 1: the differential form ds/dtau = -(Delta s + S[s]) (Eq. smud)
// marched from s(0) = 0 by one explicit Runge-Kutta step per grid interval,
// every instance of the batch at once, in FP64.  The paper names RK1 / RK2 /
// RK4 without printing their tableaux; they are read as forward Euler, Heun's
// method and the classical four-stage method.  Each stage evaluates the S
// kernel on one tau slice per instance through the engine; Omega_CC is then
// integrated from the energies at every grid point with the quadrature
// weights g (Eq. Ecc), as in the integral form.
ftcc_status rk_solve(Batch& B) {
  static const double kA1[1][3] = {{0, 0, 0}}, kB1[1] = {1.0};
  static const double kA2[2][3] = {{0, 0, 0}, {1.0, 0, 0}}, kB2[2] = {0.5, 0.5};
  static const double kA4[4][3] = {{0, 0, 0}, {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 1.0}},
                      kB4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  int ns;
  const double(*A)[3];
  const double* bw;
  switch (B.quad) {
    case FTCC_QUAD_RK1: ns = 1, A = kA1, bw = kB1; break;
    case FTCC_QUAD_RK2: ns = 2, A = kA2, bw = kB2; break;
    case FTCC_QUAD_RK4: ns = 4, A = kA4, bw = kB4; break;
    default: throw Fail{FTCC_ERR_STATE, "not an RK quadrature"};
  }
  ftcc_ctx* h = B.home;
  cudaStream_t st = h->st;
  Solver<double>& s = make_solver<double>(B, GEMM_F64);
  B.active = 0;
  const int nz = B.nz, ng = B.ng, no = B.no, nv = B.nv;
  const long long n1 = static_cast<long long>(no) * nv, n2 = n1 * no * nv;
  // stage inputs and stage derivatives, [nz][n] each; released on every exit
  struct Held {
    ftcc_ctx* h;
    Buf b[10];
    ~Held() {
      for (Buf& x : b) h->put(x);
    }
  } held{h, {}};
  Buf &Y1 = held.b[0], &Y2 = held.b[1];
  ensure(h, Y1, nz * n1 * sizeof(double));
  ensure(h, Y2, nz * n2 * sizeof(double));
  double *K1[4], *K2[4];
  for (int j = 0; j < ns; ++j) {
    ensure(h, held.b[2 + j], nz * n1 * sizeof(double));
    ensure(h, held.b[6 + j], nz * n2 * sizeof(double));
    K1[j] = static_cast<double*>(held.b[2 + j].p);
    K2[j] = static_cast<double*>(held.b[6 + j].p);
  }
  double* t1 = static_cast<double*>(s.t1.p);
  double* t2 = static_cast<double*>(s.t2.p);
  double* S1 = static_cast<double*>(s.S1.p);
  double* S2 = static_cast<double*>(s.S2.p);
  double* y1 = static_cast<double*>(Y1.p);
  double* y2 = static_cast<double*>(Y2.p);
  const double* hz = static_cast<const double*>(B.hz.p);   // [nz] steps, then [nz] betas
  const double* eps = static_cast<const double*>(B.epsz.p);
  const int* iO = static_cast<const int*>(B.idxO.p);
  const int* iV = static_cast<const int*>(B.idxV.p);
  CU(cudaMemsetAsync(t1, 0, static_cast<size_t>(nz) * ng * n1 * sizeof(double), st));   // s(tau_0) = 0
  CU(cudaMemsetAsync(t2, 0, static_cast<size_t>(nz) * ng * n2 * sizeof(double), st));
  for (int k = 0; k + 1 < ng; ++k) {
    const double* b1 = t1 + k * n1;   // s(tau_k), instance stride ng n
    const double* b2 = t2 + k * n2;
    for (int q = 0; q < ns; ++q) {
      RkTerms<double> r1{}, r2{};
      for (int j = 0; j < q; ++j)
        if (A[q][j] != 0.0) {
          r1.c[r1.n] = A[q][j], r1.K[r1.n++] = K1[j];
          r2.c[r2.n] = A[q][j], r2.K[r2.n++] = K2[j];
        }
      CU(launch_rk_combine<double>(y1, n1, b1, ng * n1, r1, hz, n1, nz, st));
      CU(launch_rk_combine<double>(y2, n2, b2, ng * n2, r2, hz, n2, nz, st));
      s.s_kernel(y1, y2, S1, S2, 1);
      CU(launch_rk_deriv<double>(K1[q], y1, S1, eps, iO, iV, B.N, no, nv, 2, nz, st));
      CU(launch_rk_deriv<double>(K2[q], y2, S2, eps, iO, iV, B.N, no, nv, 4, nz, st));
    }
    RkTerms<double> r1{}, r2{};
    for (int q = 0; q < ns; ++q) {
      r1.c[r1.n] = bw[q], r1.K[r1.n++] = K1[q];
      r2.c[r2.n] = bw[q], r2.K[r2.n++] = K2[q];
    }
    CU(launch_rk_combine<double>(t1 + (k + 1) * n1, ng * n1, b1, ng * n1, r1, hz, n1, nz, st));
    CU(launch_rk_combine<double>(t2 + (k + 1) * n2, ng * n2, b2, ng * n2, r2, hz, n2, nz, st));
  }
  CU(launch_rk_energy<double>(t1, t2, static_cast<const double*>(B.F64.p), static_cast<const double*>(B.V64.p), ng, no,
                              nv, nz, s.nb1, s.nb2, static_cast<double*>(s.part1.p), static_cast<double*>(s.part2.p),
                              st));
  CU(launch_reduce(static_cast<const double*>(s.part1.p), s.nb1, static_cast<const double*>(s.part2.p), s.nb2, ng, nz,
                   hz, static_cast<const int*>(B.live.p), static_cast<double*>(B.state.p), st));
  check_device_error(h);
  std::vector<double> sv = read_states(B);
  B.iterations = ng - 1;   // steps marched
  bool finite = true;
  for (int z = 0; z < nz; ++z) {
    const double om = sv[static_cast<size_t>(z) * kStateStride];
    if (std::isfinite(om)) B.inst[z].conv_iter = ng - 1;
    else finite = false;
  }
  if (!finite) return fail(h, FTCC_ERR_DIVERGED, "the RK march became non-finite (a step too long for the stiffness)");
  return FTCC_OK;
}

// The fixed-point loop of one batch as a state machine advanced one
// iteration at a time, so that the batches of a batched solve (one per
// orbital count) run their iterations in lockstep, each on its own stream,
// and overlap on the GPU.  Phases: the low-precision phase (TF32, then the
// BF16X3 polish) or the FP64 iteration, then the FP64 residual corrections.
struct SolveDriver {
  Batch& B;
  const ftcc_options& o;
  ftcc_ctx* h;
  std::vector<double> s, best;
  std::vector<int> stall;
  bool conv = false, finished = false, refining = false;
  int it = 0, r = 0;
  ftcc_status status = FTCC_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  double* pin = nullptr;   // the home context's pinned state copy (nullptr: read back after the wait)

  SolveDriver(Batch& b, bool pinned) : B(b), o(b.opt), h(b.home), best(b.nz, 1e300), stall(b.nz, 0) {
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    CU(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
    const size_t need = static_cast<size_t>(B.nz) * kStateStride;
    if (pinned) {
      if (h->pin_state_n < need) {
        if (h->pin_state) CU(cudaFreeHost(h->pin_state));
        h->pin_state = nullptr;
        h->pin_state_n = 0;
        CU(cudaMallocHost(&h->pin_state, need * sizeof(double)));
        h->pin_state_n = need;
      }
      pin = h->pin_state;
    }
    if (o.max_iter <= 0) end();
  }
  ~SolveDriver() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e2) cudaEventDestroy(e2);
  }
  // enqueue one iteration on the batch's stream, and the copy of its state
  // to pinned host memory behind it (no host wait)
  void launch() {
    CU(cudaEventRecord(e0, h->st));
    run_batch(B, 1);
    CU(cudaEventRecord(e1, h->st));
    if (pin)
      CU(cudaMemcpyAsync(pin, B.state.p, static_cast<size_t>(B.nz) * kStateStride * sizeof(double),
                         cudaMemcpyDeviceToHost, h->st));
    CU(cudaEventRecord(e2, h->st));
  }
  // after a grouped step (its state already in pinned memory): the
  // convergence and phase logic
  void collect_grouped(float ms) {
    B.ms_total += ms;
    B.ms_count += 1;
    s.assign(pin, pin + static_cast<size_t>(B.nz) * kStateStride);
    step();
  }
  // wait for it, then the convergence and phase logic
  void collect() {
    CU(cudaEventSynchronize(e2));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    B.ms_total += ms;
    B.ms_count += 1;
    if (pin) s.assign(pin, pin + static_cast<size_t>(B.nz) * kStateStride);
    else s = read_states(B);
    step();
  }
  bool all_done(double tol_o, double tol_a) {
    bool all = true;
    for (int z = 0; z < B.nz; ++z) {
      if (!B.live_host[z]) continue;
      const double* q = s.data() + static_cast<size_t>(z) * kStateStride;
      const bool ok = q[1] < tol_o && q[2] < tol_a;
      if (ok && B.inst[z].conv_iter < 0) B.inst[z].conv_iter = B.iterations;
      all = all && ok;
    }
    return all;
  }
  bool mixed_done(double tol) {
    bool all = true;
    for (int z = 0; z < B.nz; ++z)
      if (B.live_host[z]) all = all && s[static_cast<size_t>(z) * kStateStride + 1] < tol;
    return all;
  }
  // an instance whose Omega_CC or amplitudes stop being finite is frozen
  // (its slice keeps its last state) so that the rest of the batch goes on;
  // returns false when no live instance is left
  bool finite() {
    bool changed = false, any = false;
    for (int z = 0; z < B.nz; ++z) {
      if (!B.live_host[z]) continue;
      const double* q = s.data() + static_cast<size_t>(z) * kStateStride;
      if (!std::isfinite(q[0]) || !std::isfinite(q[2]) || std::fabs(q[0]) > 1e12) {
        B.live_host[z] = 0;
        changed = true;
      } else {
        any = true;
      }
    }
    if (changed)
      CU(cudaMemcpyAsync(B.live.p, B.live_host.data(), B.nz * sizeof(int), cudaMemcpyHostToDevice, h->st));
    return any;
  }
  void end() {
    finished = true;
    check_device_error(h);
    int dead = 0;
    for (int z = 0; z < B.nz; ++z) dead += !B.live_host[z];
    B.solved = conv && dead == 0;
    B.solved_live = conv && dead < B.nz;
    if (dead) status = fail(h, FTCC_ERR_DIVERGED, "%d of %d instances diverged (frozen)", dead, B.nz);
    else if (!conv) status = fail(h, FTCC_ERR_NOT_CONVERGED, "not converged after %d iterations", B.iterations);
  }
  void step() {
    if (refining) {
      // FP64 residual corrections: s <- s + r with the FP64 residual
      // r = Phi(s) - s (one FP64 application of the fixed-point map each), at
      // most refine_max_iter of them; they stop early once the FP64 tolerances
      // hold.  The mixed solve counts as converged when the last correction
      // moved Omega_CC by less than tol_refine.
      B.refine_iterations++;
      if (!finite()) {
        finished = true;
        status = fail(h, FTCC_ERR_DIVERGED, "Omega_CC became non-finite in refinement");
        return;
      }
      if (B.nz == 1 && !B.live_host[0]) return end();
      if (all_done(o.tol_omega, o.tol_amp)) {
        conv = true;
        return end();
      }
      if (++r < o.refine_max_iter) return;
      conv = mixed_done(o.tol_refine);
      if (conv)
        for (Inst& I : B.inst)
          if (I.conv_iter < 0) I.conv_iter = B.iterations;
      return end();
    }
    ++it;
    if (!finite()) {
      check_device_error(h);
      finished = true;
      status = fail(h, FTCC_ERR_DIVERGED, "Omega_CC became non-finite at iteration %d", B.iterations);
      return;
    }
    if (B.active == 0) {
      if (all_done(o.tol_omega, o.tol_amp)) conv = true;
      if (conv || it >= o.max_iter) end();
      return;
    }
    // a low-precision phase hands over once every instance's dOmega is small
    // or has stopped falling (or the polishing phase reached its cap)
    if (B.s32->gk == GEMM_BF16X3 && B.polishing) B.polish_iterations++;
    bool handover = true;
    for (int z = 0; z < B.nz; ++z) {
      if (!B.live_host[z]) continue;
      const double d = s[static_cast<size_t>(z) * kStateStride + 1];
      if (d < best[z]) {
        best[z] = d;
        stall[z] = 0;
      } else {
        ++stall[z];
      }
      // TF32 stops helping once Omega_CC changes by less than its unit
      // roundoff (2^-11) relative to Omega_CC
      const double floor_tf32 =
          B.s32->gk == GEMM_TF32 ? std::ldexp(std::fabs(s[static_cast<size_t>(z) * kStateStride]), -11) : 0.0;
      handover = handover && (d < o.tol_mixed || d < floor_tf32 || stall[z] >= 3);
    }
    if (B.polishing && B.polish_iterations >= o.polish_max_iter) handover = true;
    if (!handover) {
      if (it >= o.max_iter) end();
      return;
    }
    // TF32 phase done: polish with the two-way bf16 split (about 2^-16
    // relative per product against 2^-11 for TF32) from the TF32 amplitudes
    if (B.s32->gk == GEMM_TF32 && o.polish_max_iter > 0) {
      check_device_error(h);
      B.s32->set_kind(GEMM_BF16X3);
      B.polishing = true;
      std::fill(best.begin(), best.end(), 1e300);
      std::fill(stall.begin(), stall.end(), 0);
      if (it >= o.max_iter) end();
      return;
    }
    if (o.refine_max_iter == 0) {
      conv = mixed_done(o.tol_mixed);
      return end();
    }
    check_device_error(h);
    promote_to_fp64(B);
    for (Inst& I : B.inst) I.conv_iter = -1;
    refining = true;
    r = 0;
  }
};

ftcc_status solve_batch(Batch& B) {
  if (B.quad != FTCC_QUAD_SIMPSON) return rk_solve(B);
  SolveDriver d(B, true);
  while (!d.finished) {
    d.launch();
    d.collect();
  }
  return d.status;
}

// The captured iteration of a batch's current solver, if a step of it can
// run inside a graph of many batches (captured, not profiling).
cudaGraph_t step_graph(Batch& B, unsigned* gen) {
  if (!B.opt.use_graph) return nullptr;
  if (B.active == 1) {
    if (!B.s32 || !B.s32->gexec || B.s32->profiling) return nullptr;
    *gen = B.s32->graph_gen;
    return B.s32->graph;
  }
  if (!B.s64 || !B.s64->gexec || B.s64->profiling) return nullptr;
  *gen = B.s64->graph_gen;
  return B.s64->graph;
}

// One step of several batches as one graph launch: every member's captured
// iteration as a child node, each followed by the copy of its convergence
// state to the pinned host memory of its home context.  The graph is rebuilt
// when the members or one of their iterations change (a batch finished, or
// switched precision); between rebuilds a step is one cudaGraphLaunch and one
// wait, where one launch, copy and wait per batch made the host the bound of
// a step of many small instances.
struct GroupStep {
  std::vector<SolveDriver*> members;
  std::vector<std::pair<cudaGraph_t, unsigned>> keys;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr, done = nullptr;
  bool broken = false;   // building failed once: batches launch on their own
  ~GroupStep() {
    if (exec) cudaGraphExecDestroy(exec);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (done) cudaEventDestroy(done);
  }
  bool ready(const std::vector<SolveDriver*>& ms, const std::vector<std::pair<cudaGraph_t, unsigned>>& ks) {
    if (exec && ms == members && ks == keys) return true;
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    members.clear();
    keys.clear();
    if (!t0 && (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess ||
                cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess))
      return false;
    cudaGraph_t P = nullptr;
    if (cudaGraphCreate(&P, 0) != cudaSuccess) return false;
    bool ok = true;
    for (size_t k = 0; ok && k < ms.size(); ++k) {
      cudaGraphNode_t c = nullptr, cp = nullptr;
      ok = cudaGraphAddChildGraphNode(&c, P, nullptr, 0, ks[k].first) == cudaSuccess &&
           cudaGraphAddMemcpyNode1D(&cp, P, &c, 1, ms[k]->pin, ms[k]->B.state.p,
                                    static_cast<size_t>(ms[k]->B.nz) * kStateStride * sizeof(double),
                                    cudaMemcpyDeviceToHost) == cudaSuccess;
    }
    ok = ok && cudaGraphInstantiate(&exec, P, 0) == cudaSuccess;
    cudaGraphDestroy(P);
    if (!ok) {
      if (exec) cudaGraphExecDestroy(exec);
      exec = nullptr;
      cudaGetLastError();   // (the failure is reported by falling back, not as a sticky error)
      return false;
    }
    members = ms;
    keys = ks;
    return true;
  }
};

// The batches of one batched solve advanced together.  With at least
// kGroupMinBatches batches, once every unfinished batch has captured its
// iteration a step of all of them is one graph (GroupStep); before that, or
// for a batch that cannot join (no pinned state copy, profiling, no graph),
// a batch steps on its own stream.
constexpr int kGroupMinBatches = 8;
std::vector<ftcc_status> solve_batches(const std::vector<Batch*>& Bs) {
  std::vector<ftcc_status> st(Bs.size(), FTCC_OK);
  std::vector<std::unique_ptr<SolveDriver>> ds;
  for (size_t k = 0; k < Bs.size(); ++k) {
    if (Bs[k]->quad != FTCC_QUAD_SIMPSON) {
      st[k] = rk_solve(*Bs[k]);
      ds.emplace_back(nullptr);
      continue;
    }
    // the pinned state copy lives on the home context: two batches with one
    // home (never made by the batching, but possible) read back unpinned
    bool shared = false;
    for (size_t q = 0; q < k; ++q) shared = shared || Bs[q]->home == Bs[k]->home;
    ds.emplace_back(new SolveDriver(*Bs[k], !shared));
  }
  // many small batches (the block-sparse batching makes one per instance):
  // grouped steps; a few batches (size classes of the dense batching):
  // every batch keeps one iteration in flight on its own stream, so that no
  // batch waits for the slowest of the others
  int npinned = 0;
  for (auto& d : ds)
    if (d && d->pin) ++npinned;
  if (npinned < kGroupMinBatches) {
    for (auto& d : ds)
      if (d && !d->finished) d->launch();
    for (;;) {
      bool any = false;
      for (auto& d : ds)
        if (d && !d->finished) {
          any = true;
          d->collect();
          if (!d->finished) d->launch();
        }
      if (!any) break;
    }
    for (size_t k = 0; k < ds.size(); ++k)
      if (ds[k]) st[k] = ds[k]->status;
    return st;
  }
  GroupStep grp;
  for (;;) {
    std::vector<SolveDriver*> solo, grouped;
    std::vector<std::pair<cudaGraph_t, unsigned>> keys;
    for (auto& d : ds) {
      if (!d || d->finished) continue;
      unsigned gen = 0;
      cudaGraph_t g = d->pin && !grp.broken ? step_graph(d->B, &gen) : nullptr;
      if (g) {
        grouped.push_back(d.get());
        keys.emplace_back(g, gen);
      } else {
        solo.push_back(d.get());
      }
    }
    if (solo.empty() && grouped.empty()) break;
    if (grouped.size() < 2 || !grp.ready(grouped, keys)) {
      if (grouped.size() >= 2) grp.broken = true;
      solo.insert(solo.end(), grouped.begin(), grouped.end());
      grouped.clear();
    }
    for (SolveDriver* d : solo) d->launch();
    if (!grouped.empty()) {
      cudaStream_t s0 = grouped[0]->h->st;
      for (SolveDriver* d : grouped) {
        if (d->h->st == s0) continue;
        CU(cudaEventRecord(d->e1, d->h->st));   // the member's earlier work (host copies, phase changes)
        CU(cudaStreamWaitEvent(s0, d->e1, 0));
      }
      CU(cudaEventRecord(grp.t0, s0));
      CU(cudaGraphLaunch(grp.exec, s0));
      CU(cudaEventRecord(grp.t1, s0));
      CU(cudaEventRecord(grp.done, s0));
      for (SolveDriver* d : grouped) {
        d->B.iterations += 1;
        if (d->h->st != s0) CU(cudaStreamWaitEvent(d->h->st, grp.done, 0));
      }
    }
    for (SolveDriver* d : solo) d->collect();
    if (!grouped.empty()) {
      CU(cudaEventSynchronize(grp.done));
      float ms = 0;
      cudaEventElapsedTime(&ms, grp.t0, grp.t1);
      for (SolveDriver* d : grouped) d->collect_grouped(ms);
    }
  }
  for (size_t k = 0; k < ds.size(); ++k)
    if (ds[k]) st[k] = ds[k]->status;
  return st;
}

// Make the FP64 solver current with converged amplitudes (refining a
// low-precision solution in FP64 when needed).
void ensure_fp64_solution(Batch& B) {
  if (B.active == 0) return;
  promote_to_fp64(B);
  for (int r = 0; r < std::max(50, B.opt.refine_max_iter); ++r) {
    timed_iterations(B, 1);
    B.refine_iterations++;
    std::vector<double> st = read_states(B);
    bool ok = true;
    for (int z = 0; z < B.nz; ++z) {
      const double* q = st.data() + static_cast<size_t>(z) * kStateStride;
      if (B.live_host[z]) ok = ok && q[1] < B.opt.tol_omega && q[2] < B.opt.tol_amp;
    }
    if (ok) return;
  }
  throw Fail{FTCC_ERR_NOT_CONVERGED, "FP64 refinement before the adjoint did not converge"};
}

// Stationarity of the discrete Lagrangian (Eqs. Lagrangian, lmu, ltilde):
// m = -dEcc/ds - (dS/ds)^T u,  u_x = sum_y G[y,x] exp(-Delta(tau_y - tau_x)) m_y,
// with m_y = g_y lambda_y / beta; fixed-point iteration from m = 0.
// The amplitudes are fixed while this lives: the block-sparse transpose may
// keep its forward intermediates from one application to the next.
template <class T>
struct FixedAmplitudes {
  Solver<T>& s;
  explicit FixedAmplitudes(Solver<T>& s_) : s(s_) { s.vjp_fwd_reuse = true; }
  ~FixedAmplitudes() { s.vjp_fwd_reuse = false; }
};

template <class T>
int lambda_solve(Batch& B, Solver<T>& s, double tol, int max_iter) {
  s.vjp_fwd_key = nullptr;
  FixedAmplitudes<T> fixed(s);
  ftcc_ctx* h = B.home;
  constexpr size_t es = sizeof(T);
  const long long ng = B.ng, nz = B.nz;
  const long long e1 = s.n1(), e2 = s.n2();   // elements per tau point (dense or block-sparse storage)
  const long long n1 = nz * ng * e1, n2 = nz * ng * e2;
  ensure(h, B.m1, n1 * es);
  ensure(h, B.m2, n2 * es);
  ensure(h, B.mn1, n1 * es);
  ensure(h, B.mn2, n2 * es);
  ensure(h, B.u1, n1 * es);
  ensure(h, B.u2, n2 * es);
  ensure(h, B.tb1, n1 * es);
  ensure(h, B.tb2, n2 * es);
  // (the block-sparse transpose writes only the valid positions: its holes stay zero;
  // the canonical transposed propagation leaves the i = j and a = b elements of u2 zero)
  CU(cudaMemsetAsync(B.tb2.p, 0, n2 * es, h->st));
  CU(cudaMemsetAsync(B.u2.p, 0, n2 * es, h->st));
  ensure(h, B.dE1, n1 * es);
  ensure(h, B.cz, nz * ng * 8);
  const int nblk = 152 * 4;
  ensure(h, B.lpart, 4 * nblk * 8);   // [singles | doubles][block][max change, max value]
  std::vector<double> c(nz * ng);
  for (long long z = 0; z < nz; ++z)
    for (long long x = 0; x < ng; ++x) c[z * ng + x] = simpson_weight_host(static_cast<int>(x), static_cast<int>(ng)) / (ng - 1);
  CU(cudaMemcpyAsync(B.cz.p, c.data(), c.size() * 8, cudaMemcpyHostToDevice, h->st));
  CU(cudaMemsetAsync(B.m1.p, 0, n1 * es, h->st));
  CU(cudaMemsetAsync(B.m2.p, 0, n2 * es, h->st));
  CU(cudaMemsetAsync(B.mn2.p, 0, n2 * es, h->st));   // (block-sparse: only valid positions are rewritten)
  // a member frozen after diverging takes no part: its amplitudes are set to
  // zero so that its (unused) multipliers stay finite
  for (long long z = 0; z < nz; ++z)
    if (!B.live_host[z]) {
      CU(cudaMemsetAsync(static_cast<T*>(s.t1.p) + z * ng * e1, 0, ng * e1 * es, h->st));
      CU(cudaMemsetAsync(static_cast<T*>(s.t2.p) + z * ng * e2, 0, ng * e2 * es, h->st));
    }
  // dE/ds1 without the weight: f_kc + sum_jb <kj||cb> s_j^b   (Eq. E)
  s.nx = s.ng;
  T* dE1 = static_cast<T*>(B.dE1.p);
  if constexpr (sizeof(T) == 8) {
    if (s.sp)
      CU(launch_sp_fme(static_cast<const double*>(s.t1.p), s.F("zkc"), s.V("zkjcb"), s.no, s.ng, dE1, h->st));
  }
  if (!s.sp) {
    s.scatter(dE1, "zxkc", s.F("zkc"), "zkc", 1.0, 0.0, "");
    s.contract({dE1, "zxkc"}, 1.0, Tn<const T>{s.V("zkjcb"), "zkjcb", true},
               Tn<const T>{static_cast<const T*>(s.t1.p), "zxjb"});
  }
  CU(cudaStreamSynchronize(h->st));
  PropArgs a1 = prop_args(B, 2), a2 = prop_args(B, 4);
  a1.nblocks = std::max(1, std::min(prop_blocks(), static_cast<int>((a1.size + 127) / 128)));
  a2.nblocks = std::max(1, std::min(prop_blocks(), static_cast<int>((a2.size + 127) / 128)));
  std::vector<double> parts(4 * nblk);
  int it = 0, stall = 0;
  double best_rel = 1e300;
  for (it = 1; it <= max_iter; ++it) {
    CU(launch_propagate_t(static_cast<const T*>(B.m1.p), static_cast<T*>(B.u1.p), a1, h->st));
    CU(launch_propagate_t(static_cast<const T*>(B.m2.p), static_cast<T*>(B.u2.p), a2, h->st));
    for (int x0 = 0; x0 < s.ng; x0 += s.nxc) {
      const int nx = std::min(s.nxc, s.ng - x0);
      const long long f1 = x0 * e1, f2 = x0 * e2;
      s.vjp(static_cast<const T*>(s.t1.p) + f1, static_cast<const T*>(s.t2.p) + f2,
            static_cast<T*>(B.u1.p) + f1, static_cast<T*>(B.u2.p) + f2, static_cast<T*>(B.tb1.p) + f1,
            static_cast<T*>(B.tb2.p) + f2, nx);
    }
    double dmax = 0, smax = 0;
    double* lp = static_cast<double*>(B.lpart.p);
    CU(launch_lambda_combine<T, T>(dE1, static_cast<const T*>(B.tb1.p), static_cast<T*>(B.mn1.p),
                                   static_cast<const T*>(B.m1.p), e1, static_cast<int>(ng), static_cast<int>(nz),
                                   static_cast<const double*>(B.cz.p), 0.0, lp, nblk, h->st));
    CU(launch_lambda_combine<T, double>(static_cast<const double*>(B.V64.p), static_cast<const T*>(B.tb2.p),
                                        static_cast<T*>(B.mn2.p), static_cast<const T*>(B.m2.p), e2,
                                        static_cast<int>(ng), static_cast<int>(nz),
                                        static_cast<const double*>(B.cz.p), 0.25, lp + 2 * nblk, nblk, h->st,
                                        s.sp ? static_cast<const int*>(B.vall.p) : nullptr, s.sp ? B.nvall : 0));
    // one read-back of both maxima per iteration
    CU(cudaMemcpyAsync(parts.data(), lp, 4 * nblk * 8, cudaMemcpyDeviceToHost, h->st));
    sync(h);
    for (int b = 0; b < 2 * nblk; ++b) {
      dmax = std::max(dmax, parts[2 * b]);
      smax = std::max(smax, parts[2 * b + 1]);
    }
    std::swap(B.m1, B.mn1);
    std::swap(B.m2, B.mn2);
    if (!std::isfinite(dmax)) throw Fail{FTCC_ERR_DIVERGED, "lambda iteration diverged"};
    const double rel = dmax / std::max(1.0, smax);
    if (rel < tol) break;
    // in FP32 the change stops falling at the rounding of the multipliers:
    // three iterations without a new smallest change end the sweep there
    if (sizeof(T) == 4) {
      if (rel < best_rel) {
        best_rel = rel;
        stall = 0;
      } else if (++stall >= 3 && best_rel < 1e-4) {
        break;
      }
    }
  }
  check_device_error(h);
  B.lambda_iterations = it;
  B.lambda_done = it <= max_iter;
  return it;
}

// Response of the converged solve from the multipliers m (App. B): partial
// derivatives of the Lagrangian at fixed (s, m) through the thermal integral
// blocks (Fermi factors and the Fock matrix), the propagator (Delta, beta)
// and the reference (Omega0, Omega1).  Fills out[z] and rdm[z] (N x N,
// rdm[q][p] pairs with X[p][q]).
template <class T>
void response(Batch& B, Solver<T>& s, std::vector<ftcc_adjoint_result>& out, std::vector<std::vector<double>>& rdm) {
  FixedAmplitudes<T> fixed(s);
  ftcc_ctx* h = B.home;
  const int nz = B.nz, no = B.no, nv = B.nv, N = B.N, ng = B.ng;
  const long long n1 = static_cast<long long>(nz) * ng * no * nv;
  PropArgs a1 = prop_args(B, 2), a2 = prop_args(B, 4);
  a1.nblocks = std::max(1, std::min(prop_blocks(), static_cast<int>((a1.size + 127) / 128)));
  a2.nblocks = std::max(1, std::min(prop_blocks(), static_cast<int>((a2.size + 127) / 128)));
  // cotangent of S at the converged multipliers
  CU(launch_propagate_t(static_cast<const T*>(B.m1.p), static_cast<T*>(B.u1.p), a1, h->st));
  CU(launch_propagate_t(static_cast<const T*>(B.m2.p), static_cast<T*>(B.u2.p), a2, h->st));
  for (auto& kv : s.fixed_bar) h->put(kv.second);
  s.fixed_bar.clear();
  s.want_fixed_bar = true;
  for (int x0 = 0; x0 < s.ng; x0 += s.nxc) {
    const int nx = std::min(s.nxc, s.ng - x0);
    const long long f1 = static_cast<long long>(x0) * s.n1(), f2 = static_cast<long long>(x0) * s.n2();
    s.vjp(static_cast<const T*>(s.t1.p) + f1, static_cast<const T*>(s.t2.p) + f2,
          static_cast<T*>(B.u1.p) + f1, static_cast<T*>(B.u2.p) + f2, static_cast<T*>(B.tb1.p) + f1,
          static_cast<T*>(B.tb2.p) + f2, nx);
  }
  s.want_fixed_bar = false;
  // direct dependence of Omega_CC = sum_y (g_y / beta) E_y on f_ia and <ij||ab> (Eq. E)
  s.nx = s.ng;
  using CT = Tn<const T>;
  // the energy weights c_x = g_x / beta in the amplitude type
  Buf czT = h->get(static_cast<size_t>(nz) * ng * sizeof(T));
  if (!czT.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
  CU(launch_convert<double, T>(static_cast<const double*>(B.cz.p), static_cast<T*>(czT.p),
                               static_cast<long long>(nz) * ng, h->st));
  const T* cz = static_cast<const T*>(czT.p);
  const T* t1 = static_cast<const T*>(s.t1.p);
  const T* t2 = static_cast<const T*>(s.t2.p);
  T* Aov = s.fixed_adjoint(s.F("zia"));
  T* Aoovv = s.fixed_adjoint(s.V("zijab"));
  if (s.sp) {
    if constexpr (sizeof(T) == 8)
      CU(launch_sp_energy_bar(t1, t2, static_cast<const double*>(B.cz.p), static_cast<const int16_t*>(B.imp.p), N, ng,
                              Aoovv, Aov, h->st));
  } else {
    T* cs1 = static_cast<T*>(B.tb1.p);
    s.contract({Aov, "zia"}, 1.0, CT{cz, "zx"}, CT{t1, "zxia"});
    s.contract({Aoovv, "zijab"}, 0.25, CT{cz, "zx"}, CT{t2, "zxijab"});
    s.contract({cs1, "zxia"}, 1.0, CT{cz, "zx"}, CT{t1, "zxia"}, "", 0.0);
    s.contract({Aoovv, "zijab"}, 0.5, CT{cs1, "zxia"}, CT{t1, "zxjb"});
  }
  (void)n1;
  // per-orbital sums through the Fermi factors
  Buf Do = h->get(static_cast<size_t>(nz) * no * 8), Dv = h->get(static_cast<size_t>(nz) * nv * 8);
  Buf Fbar = h->get(static_cast<size_t>(nz) * N * N * 8), Gn = h->get(static_cast<size_t>(nz) * N * 8);
  Buf Ee = h->get(static_cast<size_t>(nz) * N * 8), Eb = h->get(static_cast<size_t>(nz) * 8);
  if (!Do.p || !Dv.p || !Fbar.p || !Gn.p || !Ee.p || !Eb.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
  CU(cudaMemsetAsync(Do.p, 0, Do.bytes, h->st));
  CU(cudaMemsetAsync(Dv.p, 0, Dv.bytes, h->st));
  CU(cudaMemsetAsync(Fbar.p, 0, Fbar.bytes, h->st));
  CU(cudaMemsetAsync(Ee.p, 0, Ee.bytes, h->st));
  CU(cudaMemsetAsync(Eb.p, 0, Eb.bytes, h->st));
  // block-sparse storage: the Fock blocks are diagonals; their I * Ibar (two
  // slots, both orbital p) and their scatter to Fbar (the diagonal) are done
  // on the host
  std::vector<double> spDo(s.sp ? N : 0, 0.0), spDv(s.sp ? N : 0, 0.0);
  if (s.sp) {
    if constexpr (sizeof(T) == 8) {
      for (auto& kv : s.Vb) {
        auto it = s.fixed_bar.find(kv.second.p);
        if (it == s.fixed_bar.end()) continue;
        int cls = 0;
        for (int k = 0; k < 4; ++k)
          if (kv.first[k] == 'v') cls |= 1 << k;
        CU(launch_sp_slot_sums(static_cast<const double*>(kv.second.p), static_cast<const double*>(it->second.p),
                               static_cast<const int16_t*>(B.imp.p), N, cls, static_cast<double*>(Do.p),
                               static_cast<double*>(Dv.p), h->st));
      }
      std::vector<double> fb(N), fv(N), Fh(static_cast<size_t>(N) * N, 0.0);
      const Inst& I0 = B.inst[0];
      for (auto& kv : s.Fb) {
        auto it = s.fixed_bar.find(kv.second.p);
        if (it == s.fixed_bar.end()) continue;
        CU(cudaMemcpyAsync(fb.data(), it->second.p, N * 8, cudaMemcpyDeviceToHost, h->st));
        CU(cudaMemcpyAsync(fv.data(), kv.second.p, N * 8, cudaMemcpyDeviceToHost, h->st));
        sync(h);
        for (int p = 0; p < N; ++p) {
          const double prod = fb[p] * fv[p];
          for (int k = 0; k < 2; ++k) (kv.first[k] == 'o' ? spDo : spDv)[p] += prod;
          double f = 1.0;
          for (int k = 0; k < 2; ++k) f *= std::sqrt(kv.first[k] == 'o' ? I0.n_host[p] : I0.nbar_host[p]);
          Fh[static_cast<size_t>(p) * N + p] += fb[p] * f;
        }
      }
      CU(cudaMemcpyAsync(Fbar.p, Fh.data(), Fh.size() * 8, cudaMemcpyHostToDevice, h->st));
      sync(h);
    }
  }
  for (auto* mp : {&s.Vb, &s.Fb}) {
    if (s.sp) break;
    for (auto& kv : *mp) {
      auto it = s.fixed_bar.find(kv.second.p);
      if (it == s.fixed_bar.end()) continue;
      const std::string& pat = kv.first;
      int dims[4], cls = 0;
      for (size_t k = 0; k < pat.size(); ++k) {
        dims[k] = pat[k] == 'o' ? no : nv;
        if (pat[k] == 'v') cls |= 1 << k;
      }
      CU(launch_slot_sums(static_cast<const T*>(kv.second.p), static_cast<const T*>(it->second.p),
                          static_cast<int>(pat.size()), dims, cls, no, nv, nz, static_cast<double*>(Do.p),
                          static_cast<double*>(Dv.p), h->st));
      if (pat.size() == 2) {
        const bool h0 = pat[0] == 'o', h1 = pat[1] == 'o';
        CU(launch_fbar_scatter(static_cast<const T*>(it->second.p), h0 ? no : nv, h1 ? no : nv,
                               static_cast<const int*>(h0 ? B.idxO.p : B.idxV.p),
                               static_cast<const double*>(h0 ? B.facOz.p : B.facVz.p), h0 ? no : nv,
                               static_cast<const int*>(h1 ? B.idxO.p : B.idxV.p),
                               static_cast<const double*>(h1 ? B.facOz.p : B.facVz.p), h1 ? no : nv, N, nz,
                               static_cast<double*>(Fbar.p), h->st));
      }
    }
  }
  for (int z = 0; z < nz; ++z)
    CU(launch_fock_n(static_cast<const double*>(Fbar.p) + static_cast<long long>(z) * N * N,
                     static_cast<const double*>(B.inst[z].ctx->eri.p), N, static_cast<double*>(Gn.p) + z * N, h->st));
  CU(launch_prop_response(static_cast<const T*>(s.S1.p), static_cast<const T*>(B.m1.p),
                          static_cast<const double*>(B.epsz.p), a1, static_cast<double*>(Ee.p),
                          static_cast<double*>(Eb.p), h->st));
  CU(launch_prop_response(static_cast<const T*>(s.S2.p), static_cast<const T*>(B.m2.p),
                          static_cast<const double*>(B.epsz.p), a2, static_cast<double*>(Ee.p),
                          static_cast<double*>(Eb.p), h->st));
  std::vector<double> hDo(nz * no), hDv(nz * nv), hF(static_cast<size_t>(nz) * N * N), hGn(nz * N), hEe(nz * N), hEb(nz);
  CU(cudaMemcpyAsync(hDo.data(), Do.p, Do.bytes, cudaMemcpyDeviceToHost, h->st));
  CU(cudaMemcpyAsync(hDv.data(), Dv.p, Dv.bytes, cudaMemcpyDeviceToHost, h->st));
  CU(cudaMemcpyAsync(hF.data(), Fbar.p, Fbar.bytes, cudaMemcpyDeviceToHost, h->st));
  CU(cudaMemcpyAsync(hGn.data(), Gn.p, Gn.bytes, cudaMemcpyDeviceToHost, h->st));
  CU(cudaMemcpyAsync(hEe.data(), Ee.p, Ee.bytes, cudaMemcpyDeviceToHost, h->st));
  CU(cudaMemcpyAsync(hEb.data(), Eb.p, Eb.bytes, cudaMemcpyDeviceToHost, h->st));
  sync(h);
  for (size_t p = 0; p < spDo.size(); ++p) {
    hDo[p] += spDo[p];
    hDv[p] += spDv[p];
  }
  const std::vector<double> st = read_states(B);
  std::vector<double> eps(N), fdiag(N * N), hdiag(N * N);
  out.assign(nz, ftcc_adjoint_result{});
  rdm.assign(nz, std::vector<double>(static_cast<size_t>(N) * N, 0.0));
  for (int z = 0; z < nz; ++z) {
    const Inst& I = B.inst[z];
    CU(cudaMemcpyAsync(eps.data(), I.ctx->eps.p, N * 8, cudaMemcpyDeviceToHost, h->st));
    CU(cudaMemcpyAsync(fdiag.data(), I.f.p, static_cast<size_t>(N) * N * 8, cudaMemcpyDeviceToHost, h->st));
    sync(h);
    std::vector<int> posO(N, -1), posV(N, -1);
    for (int k = 0; k < no; ++k) posO[B.O[k]] = k;
    for (int k = 0; k < nv; ++k) posV[B.V[k]] = k;
    const double beta = I.beta, mu = I.mu;
    double dmu = 0, dbeta = 0, sum_n = 0, sum_ne = 0;
    std::vector<double> Tq(N);
    for (int q = 0; q < N; ++q) {
      const double nq = I.n_host[q], nb = I.nbar_host[q];
      const double Do_q = posO[q] >= 0 ? hDo[z * no + posO[q]] : 0.0;
      const double Dv_q = posV[q] >= 0 ? hDv[z * nv + posV[q]] : 0.0;
      const double Ln = (fdiag[static_cast<size_t>(q) * N + q] - eps[q]) + hGn[z * N + q];
      Tq[q] = Ln * nq * nb + 0.5 * Do_q * nb - 0.5 * Dv_q * nq;   // dL/dz'_q, z'_q = -beta (eps_q - mu)
      sum_n += nq;
      sum_ne += nq * (eps[q] - mu);
      dmu += beta * Tq[q];
      dbeta += -(eps[q] - mu) * Tq[q];
    }
    const double omega0 = I.omega0;
    dmu += -sum_n;
    dbeta += -omega0 / beta + sum_ne / beta + hEb[z] / beta;
    const double* F = hF.data() + static_cast<size_t>(z) * N * N;
    std::vector<double>& R = rdm[z];
    for (int p = 0; p < N; ++p)
      for (int q = 0; q < N; ++q) R[static_cast<size_t>(q) * N + p] = F[static_cast<size_t>(p) * N + q];
    double tr = 0;
    for (int q = 0; q < N; ++q) {
      R[static_cast<size_t>(q) * N + q] = I.n_host[q] - beta * Tq[q] + hEe[z * N + q];
      tr += R[static_cast<size_t>(q) * N + q];
    }
    const double omega = I.omega0 + I.omega1 + st[static_cast<size_t>(z) * kStateStride];
    ftcc_adjoint_result& r = out[z];
    r.dOmega_dmu = dmu;
    r.dOmega_dbeta = dbeta;
    r.N = -dmu;
    r.E = omega + beta * dbeta + mu * r.N;
    r.S = beta * beta * dbeta;
    r.trace_rdm1 = tr;
    r.iterations = B.lambda_iterations;
  }
  Buf* bs[] = {&Do, &Dv, &Fbar, &Gn, &Ee, &Eb, &czT};
  for (Buf* q : bs) h->put(*q);
}

ftcc_status check_solve_args(ftcc_ctx* c, double beta, double mu, int ngrid, ftcc_quadrature quad) {
  if (c->N == 0) return fail(c, FTCC_ERR_STATE, "build_integrals first");
  if (!(beta > 0) || !std::isfinite(beta) || !std::isfinite(mu) || ngrid < 3 || ngrid > 256)
    return fail(c, FTCC_ERR_INVALID_ARG, "need beta > 0 finite, mu finite, 3 <= ngrid <= 256");
  if (quad != FTCC_QUAD_SIMPSON && quad != FTCC_QUAD_RK1 && quad != FTCC_QUAD_RK2 && quad != FTCC_QUAD_RK4)
    return fail(c, FTCC_ERR_INVALID_ARG, "unknown quadrature");
  return FTCC_OK;
}

// The RK drivers march the FP64 amplitudes over the whole grid at once.
ftcc_status check_quad_options(ftcc_ctx* c, ftcc_quadrature quad, const ftcc_options& o) {
  if (quad == FTCC_QUAD_SIMPSON) return FTCC_OK;
  if (o.block_sparse) return fail(c, FTCC_ERR_UNSUPPORTED, "block_sparse: Simpson integral form only");
  if (o.precision != FTCC_PREC_FP64)
    return fail(c, FTCC_ERR_UNSUPPORTED, "the RK drivers run in FP64 (precision = FTCC_PREC_FP64)");
  if (o.stream_tau) return fail(c, FTCC_ERR_UNSUPPORTED, "the RK drivers keep every tau point (stream_tau = 0)");
  return FTCC_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

const char* ftcc_status_string(ftcc_status s) {
  const int i = static_cast<int>(s);
  if (i < 0 || i > 9) return "unknown status";
  return kStatusText[i];
}

const char* ftcc_last_error(const ftcc_ctx* c) { return c ? c->err.c_str() : "null context"; }

ftcc_status ftcc_create(int device, void* stream, const ftcc_allocator* alloc, ftcc_ctx** out) {
  if (!out) return FTCC_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return FTCC_ERR_NO_DEVICE;
  if (device < 0 || device >= n) return FTCC_ERR_INVALID_ARG;
  if (alloc && (!alloc->alloc || !alloc->release)) return FTCC_ERR_INVALID_ARG;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return FTCC_ERR_CUDA;
  if (!(prop.major == 10 && prop.minor == 3)) return FTCC_ERR_UNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) return FTCC_ERR_CUDA;
  ftcc_ctx* c = new ftcc_ctx();
  c->device = device;
  c->st = static_cast<cudaStream_t>(stream);
  if (!c->st) {
    // the legacy default stream cannot be captured into a graph: own a stream
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return FTCC_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (alloc) {
    c->alloc.a = *alloc;
    c->alloc.custom = true;
  }
  c->dev_err = static_cast<int*>(c->alloc.get(sizeof(int) * 4));
  if (!c->dev_err) {
    ftcc_destroy(c);
    return FTCC_ERR_OOM;
  }
  cudaMemsetAsync(c->dev_err, 0, sizeof(int) * 4, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) {
    ftcc_destroy(c);
    return FTCC_ERR_CUDA;
  }
  *out = c;
  return FTCC_OK;
}

void ftcc_destroy(ftcc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->st);
  // a batch whose home is this context dies with it (members lose their solve)
  if (c->batch && c->batch->home == c) {
    std::shared_ptr<Batch> b = c->batch;
    for (Inst& I : b->inst)
      if (I.ctx && I.ctx != c) I.ctx->batch.reset();
    c->batch.reset();
  }
  c->batch.reset();
  c->sptab.reset();
  if (c->pin_state) cudaFreeHost(c->pin_state);
  if (c->st2) cudaStreamDestroy(c->st2);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  c->put(c->h);
  c->put(c->eri);
  c->put(c->eps);
  if (c->dev_err) c->alloc.put(c->dev_err);
  if (c->own_stream) cudaStreamDestroy(c->st);
  delete c;
}

int ftcc_num_orbitals(const ftcc_ctx* c) { return c ? c->N : 0; }

static void drop_batch(ftcc_ctx* c) {
  if (!c->batch) return;
  std::shared_ptr<Batch> b = c->batch;
  for (Inst& I : b->inst)
    if (I.ctx) I.ctx->batch.reset();
}

ftcc_status build_integrals(ftcc_ctx* c, const ftcc_system* s) {
  if (!c || !s) return FTCC_ERR_INVALID_ARG;
  return run_guarded(c, [&]() -> ftcc_status {
    CU(cudaSetDevice(c->device));
    drop_batch(c);
    int N = 0;
    std::vector<int> nvec;
    std::vector<double> hh, he, hp;   // host-built site-basis systems
    if (s->kind == FTCC_SYS_HUBBARD_1D) {
      if (s->L < 1 || s->pbc != 1 || !std::isfinite(s->t) || !std::isfinite(s->U))
        return fail(c, FTCC_ERR_INVALID_ARG, "Hubbard: need L >= 1, pbc = 1, finite t and U");
      if (s->reference < FTCC_REF_KSPACE_RHF || s->reference > FTCC_REF_UHF_SITE)
        return fail(c, FTCC_ERR_INVALID_ARG, "Hubbard: unknown reference %d", s->reference);
      N = 2 * s->L;
      if (s->reference != FTCC_REF_KSPACE_RHF) {
        std::string msg;
        if (!hubbard_site_reference(s->L, s->t, s->U, s->reference, hh, he, hp, msg))
          return fail(c, FTCC_ERR_NOT_CONVERGED, "Hubbard reference: %s", msg.c_str());
      }
    } else if (s->kind == FTCC_SYS_UEG) {
      if (s->n_elec < 2 || (s->n_elec & 1) || !(s->rs > 0) || !std::isfinite(s->rs))
        return fail(c, FTCC_ERR_INVALID_ARG, "UEG: need an even n_elec >= 2 and rs > 0");
      if (s->n_pw < 1 || !shell_grid(s->n_pw, nvec))
        return fail(c, FTCC_ERR_INVALID_ARG, "UEG: %d plane waves is not a closed shell", s->n_pw);
      if (s->n_elec / 2 > s->n_pw) return fail(c, FTCC_ERR_INVALID_ARG, "UEG: more electrons than orbitals");
      N = 2 * s->n_pw;
    } else if (s->kind == FTCC_SYS_GENERIC) {
      if (s->N < 1 || !s->h || !s->eri || !s->eps) return fail(c, FTCC_ERR_INVALID_ARG, "generic: need N >= 1 and arrays");
      N = s->N;
    } else {
      return fail(c, FTCC_ERR_INVALID_ARG, "unknown system kind %d", s->kind);
    }
    const long long N4 = static_cast<long long>(N) * N * N * N;
    c->put(c->h);
    c->put(c->eri);
    c->put(c->eps);
    c->N = 0;
    c->sptab.reset();
    ensure(c, c->h, static_cast<size_t>(N) * N * sizeof(double));
    ensure(c, c->eri, N4 * sizeof(double));
    ensure(c, c->eps, static_cast<size_t>(N) * sizeof(double));
    if (s->kind == FTCC_SYS_HUBBARD_1D && s->reference != FTCC_REF_KSPACE_RHF) {
      CU(cudaMemcpyAsync(c->h.p, hh.data(), hh.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
      CU(cudaMemcpyAsync(c->eri.p, he.data(), he.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
      CU(cudaMemcpyAsync(c->eps.p, hp.data(), hp.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    } else if (s->kind == FTCC_SYS_HUBBARD_1D) {
      CU(launch_hubbard(static_cast<double*>(c->h.p), static_cast<double*>(c->eri.p), static_cast<double*>(c->eps.p),
                        s->L, s->t, s->U, c->st));
    } else if (s->kind == FTCC_SYS_UEG) {
      const int M = s->n_pw;
      Buf nv = c->get(nvec.size() * sizeof(int));
      if (!nv.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
      CU(cudaMemcpyAsync(nv.p, nvec.data(), nvec.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
      const double vol = 4.0 / 3.0 * M_PI * s->n_elec * s->rs * s->rs * s->rs;
      const double Lc = std::cbrt(vol);
      CU(launch_ueg(static_cast<double*>(c->h.p), static_cast<double*>(c->eri.p), static_cast<double*>(c->eps.p),
                    static_cast<const int*>(nv.p), M, s->n_elec / 2, vol, 2.0 * M_PI / Lc, c->st));
      sync(c);
      c->put(nv);
    } else {
      CU(cudaMemcpyAsync(c->h.p, s->h, static_cast<size_t>(N) * N * sizeof(double), cudaMemcpyHostToDevice, c->st));
      CU(cudaMemcpyAsync(c->eri.p, s->eri, N4 * sizeof(double), cudaMemcpyHostToDevice, c->st));
      CU(cudaMemcpyAsync(c->eps.p, s->eps, static_cast<size_t>(N) * sizeof(double), cudaMemcpyHostToDevice, c->st));
    }
    sync(c);
    // conserved orbital charges: p = sigma * L + m with crystal momentum m
    // (mod L) for the k-space ring, p = sigma * n_pw + g with the plane wave
    // n_g for the gas; S_z as sigma
    c->charge.clear();
    for (int k = 0; k < 4; ++k) c->charge_mod[k] = 0;
    if (s->kind == FTCC_SYS_HUBBARD_1D && s->reference == FTCC_REF_KSPACE_RHF) {
      for (int p = 0; p < N; ++p) c->charge.push_back({p % s->L, p / s->L, 0, 0});
      c->charge_mod[0] = s->L;
    } else if (s->kind == FTCC_SYS_UEG) {
      const int M = s->n_pw;
      for (int p = 0; p < N; ++p) {
        const int g = p % M;
        c->charge.push_back({nvec[3 * g], nvec[3 * g + 1], nvec[3 * g + 2], p / M});
      }
    } else if (s->kind == FTCC_SYS_GENERIC && s->charge) {
      for (int p = 0; p < N; ++p)
        c->charge.push_back({s->charge[4 * p], s->charge[4 * p + 1], s->charge[4 * p + 2], s->charge[4 * p + 3]});
      if (s->charge_mod)
        for (int k = 0; k < 4; ++k) c->charge_mod[k] = std::max(0, s->charge_mod[k]);
    }
    c->N = N;
    return FTCC_OK;
  });
}

ftcc_status ftcc_get_system(ftcc_ctx* c, double* eps, double* h, double* eri) {
  if (!c) return FTCC_ERR_INVALID_ARG;
  if (c->N == 0) return fail(c, FTCC_ERR_STATE, "no system built");
  return run_guarded(c, [&]() -> ftcc_status {
    const size_t N = c->N;
    if (eps) CU(cudaMemcpyAsync(eps, c->eps.p, N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (h) CU(cudaMemcpyAsync(h, c->h.p, N * N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (eri) CU(cudaMemcpyAsync(eri, c->eri.p, N * N * N * N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    sync(c);
    return FTCC_OK;
  });
}

ftcc_status ftcc_get_charges(ftcc_ctx* c, int* charge, int* charge_mod) {
  if (!c) return FTCC_ERR_INVALID_ARG;
  if (c->N == 0 || static_cast<int>(c->charge.size()) != c->N)
    return fail(c, FTCC_ERR_STATE, "the system carries no orbital charges");
  if (charge)
    for (int p = 0; p < c->N; ++p)
      for (int k = 0; k < 4; ++k) charge[4 * p + k] = c->charge[p][k];
  if (charge_mod)
    for (int k = 0; k < 4; ++k) charge_mod[k] = c->charge_mod[k];
  return FTCC_OK;
}

ftcc_status ftcc_reference_mu(ftcc_ctx* c, double beta, double n_elec, double* mu) {
  if (!c || !mu || !(beta > 0) || !std::isfinite(beta)) return FTCC_ERR_INVALID_ARG;
  if (c->N == 0) return fail(c, FTCC_ERR_STATE, "no system built");
  if (!(n_elec > 0) || !(n_elec < c->N)) return fail(c, FTCC_ERR_INVALID_ARG, "need 0 < n_elec < N");
  return run_guarded(c, [&]() -> ftcc_status {
    std::vector<double> e(c->N);
    CU(cudaMemcpyAsync(e.data(), c->eps.p, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    sync(c);
    auto count = [&](double m) {
      double s = 0;
      for (double x : e) {
        const double z = beta * (x - m);
        s += z > 0 ? std::exp(-z) / (1.0 + std::exp(-z)) : 1.0 / (1.0 + std::exp(z));
      }
      return s;
    };
    double lo = *std::min_element(e.begin(), e.end()) - 50.0 / beta - 1.0;
    double hi = *std::max_element(e.begin(), e.end()) + 50.0 / beta + 1.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(lo)); ++it) {
      const double m = 0.5 * (lo + hi);
      if (count(m) < n_elec) lo = m;
      else hi = m;
    }
    *mu = 0.5 * (lo + hi);
    return FTCC_OK;
  });
}

// mu_CC with N(mu) = -dOmega/dmu = n_target (App. D): secant steps from mu0
// and mu0 +- dmu (towards the target), regula falsi with the Illinois
// weighting once the target is straddled.  Each N(mu) is a full solve plus
// the adjoint on this context.
ftcc_status ftcc_mu_for_n(ftcc_ctx* c, double beta, double n_target, int ngrid, ftcc_quadrature quad,
                          const ftcc_options* opt, double mu0, double dmu, double tol_n, int max_evals, double* mu_out,
                          double* n_out, int* evals_out, ftcc_result* out) {
  if (!c || !mu_out || !(beta > 0) || !std::isfinite(beta) || !std::isfinite(mu0) || !(dmu > 0) ||
      !std::isfinite(dmu) || !(tol_n > 0) || max_evals < 2 || !std::isfinite(n_target))
    return FTCC_ERR_INVALID_ARG;
  if (c->N == 0) return fail(c, FTCC_ERR_STATE, "no system built");
  if (!(n_target > 0) || !(n_target < c->N)) return fail(c, FTCC_ERR_INVALID_ARG, "need 0 < n_target < N");
  int evals = 0;
  ftcc_result last{};
  auto f = [&](double m, double* val) -> ftcc_status {
    ftcc_status s = ft_ccsd_solve(c, beta, m, ngrid, quad, opt, &last);
    if (s != FTCC_OK) return s;
    ftcc_adjoint_result ar{};
    s = ft_ccsd_adjoint(c, &ar, nullptr);
    if (s != FTCC_OK) return s;
    ++evals;
    *val = ar.N - n_target;
    if (!std::isfinite(*val)) return fail(c, FTCC_ERR_DIVERGED, "N(mu) not finite at mu = %.17g", m);
    return FTCC_OK;
  };
  auto finish = [&](double m, double fm, ftcc_status s) {
    *mu_out = m;
    if (n_out) *n_out = fm + n_target;
    if (evals_out) *evals_out = evals;
    if (out) *out = last;
    return s;
  };
  double a = mu0, fa = 0.0;
  ftcc_status s = f(a, &fa);
  if (s != FTCC_OK) return s;
  if (std::fabs(fa) < tol_n) return finish(a, fa, FTCC_OK);
  double b = mu0 + (fa < 0 ? dmu : -dmu), fb = 0.0;
  if ((s = f(b, &fb)) != FTCC_OK) return s;
  bool bracket = fa * fb < 0;
  int side = 0;
  while (std::fabs(fb) >= tol_n) {
    if (evals >= max_evals)
      return finish(b, fb, fail(c, FTCC_ERR_NOT_CONVERGED, "|N - n_target| = %.3g after %d evaluations",
                                std::fabs(fb), evals));
    if (fb == fa) return finish(b, fb, fail(c, FTCC_ERR_NOT_CONVERGED, "flat N(mu): no secant step"));
    const double m = b - fb * (b - a) / (fb - fa);
    double fm = 0.0;
    if ((s = f(m, &fm)) != FTCC_OK) return s;
    if (bracket) {
      // keep the pair that straddles the target; halve the weight of an end
      // point retained twice in a row (Illinois)
      if (fm * fb < 0) {
        a = b;
        fa = fb;
        side = 0;
      } else {
        if (side == -1) fa *= 0.5;
        side = -1;
      }
      b = m;
      fb = fm;
    } else {
      a = b;
      fa = fb;
      b = m;
      fb = fm;
      bracket = fa * fb < 0;
    }
  }
  return finish(b, fb, FTCC_OK);
}

ftcc_status ftcc_prepare(ftcc_ctx* c, double beta, double mu, int ngrid, ftcc_quadrature quad, const ftcc_options* opt,
                         ftcc_result* out) {
  if (!c) return FTCC_ERR_INVALID_ARG;
  ftcc_status s = check_solve_args(c, beta, mu, ngrid, quad);
  if (s != FTCC_OK) return s;
  const ftcc_options o = opt ? *opt : default_options();
  if ((s = check_options(c, o)) != FTCC_OK) return s;
  if ((s = check_quad_options(c, quad, o)) != FTCC_OK) return s;
  return run_guarded(c, [&]() -> ftcc_status {
    drop_batch(c);
    ftcc_ctx* cs[1] = {c};
    std::shared_ptr<Batch> B = prepare_batch(cs, 1, &beta, &mu, ngrid, o);
    B->quad = quad;
    fill_result(*B, 0, read_states(*B), out);
    return FTCC_OK;
  });
}

ftcc_status ft_ccsd_iterate(ftcc_ctx* c, int n_iter, ftcc_result* out) {
  if (!c || n_iter < 0) return FTCC_ERR_INVALID_ARG;
  if (!c->batch) return fail(c, FTCC_ERR_STATE, "ftcc_prepare or ft_ccsd_solve first");
  if (c->batch->quad != FTCC_QUAD_SIMPSON)
    return fail(c, FTCC_ERR_UNSUPPORTED, "the RK drivers march the grid once (ft_ccsd_solve), they do not iterate");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    CU(cudaSetDevice(B.home->device));
    if (n_iter > 0) B.lambda_done = B.resp_done = false;   // the amplitudes move: multipliers are stale
    run_batch(B, n_iter);
    check_device_error(B.home);
    if (out) fill_result(B, c->member, read_states(B), out);
    return FTCC_OK;
  });
}

ftcc_status ft_ccsd_solve(ftcc_ctx* c, double beta, double mu, int ngrid, ftcc_quadrature quad, const ftcc_options* opt,
                          ftcc_result* out) {
  ftcc_status s = ftcc_prepare(c, beta, mu, ngrid, quad, opt, nullptr);
  if (s != FTCC_OK) return s;
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    ftcc_status r = solve_batch(B);
    fill_result(B, 0, read_states(B), out);
    return r;
  });
}

static ftcc_status batched(ftcc_ctx* const* ctx, int n, const double* beta, const double* mu, int ngrid,
                           ftcc_quadrature quad, const ftcc_options* opt, ftcc_result* out, bool iterate) {
  if (!ctx || n < 1 || !beta || !mu) return FTCC_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!ctx[i]) return FTCC_ERR_INVALID_ARG;
  ftcc_ctx* c0 = ctx[0];
  for (int i = 0; i < n; ++i) {
    ftcc_status s = check_solve_args(ctx[i], beta[i], mu[i], ngrid, quad);
    if (s != FTCC_OK) return fail(c0, s, "instance %d: %s", i, ctx[i]->err.c_str());
    if (ctx[i]->device != c0->device) return fail(c0, FTCC_ERR_INVALID_ARG, "instances on different devices");
    for (int j = 0; j < i; ++j)
      if (ctx[j] == ctx[i]) return fail(c0, FTCC_ERR_INVALID_ARG, "a context appears twice");
  }
  const ftcc_options o = opt ? *opt : default_options();
  ftcc_status s = check_options(c0, o);
  if (s != FTCC_OK) return s;
  if ((s = check_quad_options(c0, quad, o)) != FTCC_OK) return s;
  return run_guarded(c0, [&]() -> ftcc_status {
    for (int i = 0; i < n; ++i) drop_batch(ctx[i]);
    // one batch per orbital count, in order of first appearance; the batches
    // then iterate together (solve_batches).  With block_sparse every
    // instance is a batch of its own (its charge tables and sectors), each on
    // its context's stream, iterating in lockstep with the others.
    std::vector<int> done(n, 0);
    ftcc_status worst = FTCC_OK;
    std::vector<std::shared_ptr<Batch>> batches;
    std::vector<std::vector<int>> members;
    for (int i = 0; i < n; ++i) {
      if (done[i]) continue;
      std::vector<ftcc_ctx*> cs;
      std::vector<double> bs, ms;
      std::vector<int> idx;
      for (int j = i; j < n; ++j)
        if (!done[j] && ctx[j]->N == ctx[i]->N && (!o.block_sparse || j == i)) {
          cs.push_back(ctx[j]);
          bs.push_back(beta[j]);
          ms.push_back(mu[j]);
          idx.push_back(j);
          done[j] = 1;
        }
      std::shared_ptr<Batch> B = prepare_batch(cs.data(), static_cast<int>(cs.size()), bs.data(), ms.data(), ngrid, o);
      B->quad = quad;
      batches.push_back(B);
      members.push_back(idx);
    }
    if (!iterate) return FTCC_OK;
    std::vector<Batch*> raw;
    for (auto& B : batches) raw.push_back(B.get());
    const std::vector<ftcc_status> rs = solve_batches(raw);
    for (size_t b = 0; b < batches.size(); ++b) {
      Batch& B = *batches[b];
      const ftcc_status r = rs[b];
      if (r != FTCC_OK) {
        if (worst == FTCC_OK) c0->err = B.home->err;
        if (worst == FTCC_OK || r == FTCC_ERR_DIVERGED) worst = r;
      }
      const std::vector<double> st = read_states(B);
      if (out)
        for (size_t k = 0; k < members[b].size(); ++k) fill_result(B, static_cast<int>(k), st, &out[members[b][k]]);
    }
    return worst;
  });
}

ftcc_status ft_ccsd_solve_batched(ftcc_ctx* const* ctx, int n, const double* beta, const double* mu, int ngrid,
                                  ftcc_quadrature quad, const ftcc_options* opt, ftcc_result* out) {
  return batched(ctx, n, beta, mu, ngrid, quad, opt, out, true);
}

ftcc_status ftcc_prepare_batched(ftcc_ctx* const* ctx, int n, const double* beta, const double* mu, int ngrid,
                                 ftcc_quadrature quad, const ftcc_options* opt) {
  return batched(ctx, n, beta, mu, ngrid, quad, opt, nullptr, false);
}

ftcc_status ft_ccsd_adjoint(ftcc_ctx* c, ftcc_adjoint_result* out, double* rdm1) {
  if (c && c->batch && c->batch->quad != FTCC_QUAD_SIMPSON)
    return fail(c, FTCC_ERR_UNSUPPORTED, "the adjoint is built for the integral (Simpson) form only");
  if (!c) return FTCC_ERR_INVALID_ARG;
  if (!c->batch || !(c->batch->solved || (c->batch->solved_live && c->batch->live_host[c->member])))
    return fail(c, FTCC_ERR_STATE, "the adjoint needs a converged ft_ccsd_solve");
  if (c->batch->opt.stream_tau)
    return fail(c, FTCC_ERR_UNSUPPORTED, "the adjoint needs S at every tau point (solve without stream_tau)");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    CU(cudaSetDevice(B.home->device));
    std::vector<ftcc_adjoint_result>& res = B.resp;
    std::vector<std::vector<double>>& rdms = B.resp_rdm;
    if (B.resp_done) {
      // another member of a batch whose response is already known
    } else if (B.active == 1 && B.opt.mixed_adjoint && !B.sparse) {
      // the lambda sweep and the response on the FP32 solver: FP32
      // multipliers, BF16X3 contractions in the VJP, FP64 propagator
      // factors, weights and sums
      Solver<float>& s = *B.s32;
      s.set_kind(GEMM_BF16X3);
      if (!B.lambda_done) lambda_solve<float>(B, s, 1e-7, 400);
      if (!B.lambda_done) return fail(c, FTCC_ERR_NOT_CONVERGED, "lambda equations not converged");
      B.adjoint_fp32 = true;
      response<float>(B, s, res, rdms);
    } else {
      ensure_fp64_solution(B);
      if (!B.lambda_done) lambda_solve<double>(B, *B.s64, 1e-11, 400);
      if (!B.lambda_done) return fail(c, FTCC_ERR_NOT_CONVERGED, "lambda equations not converged");
      B.adjoint_fp32 = false;
      response<double>(B, *B.s64, res, rdms);
    }
    B.resp_done = true;
    if (out) *out = res[c->member];
    if (rdm1) memcpy(rdm1, rdms[c->member].data(), rdms[c->member].size() * sizeof(double));
    check_device_error(B.home);
    return FTCC_OK;
  });
}

ftcc_status ft_ccsd_adjoint_batched(ftcc_ctx* const* ctx, int n, ftcc_adjoint_result* out, ftcc_status* status) {
  if (!ctx || n < 1 || !out || !status) return FTCC_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!ctx[i]) return FTCC_ERR_INVALID_ARG;
  // members of one batch share its response: one group per batch (a context
  // without a batch is a group of its own and fails with FTCC_ERR_STATE)
  std::vector<std::vector<int>> groups;
  std::map<const Batch*, size_t> gid;
  for (int i = 0; i < n; ++i) {
    const Batch* b = ctx[i]->batch.get();
    if (b) {
      auto it = gid.find(b);
      if (it != gid.end()) {
        groups[it->second].push_back(i);
        continue;
      }
      gid.emplace(b, groups.size());
    }
    groups.push_back({i});
  }
  std::atomic<size_t> next{0};
  auto work = [&]() {
    for (size_t g; (g = next.fetch_add(1)) < groups.size();)
      for (int i : groups[g]) status[i] = ft_ccsd_adjoint(ctx[i], &out[i], nullptr);
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>(groups.size(), hw);
  std::vector<std::thread> pool;
  try {
    for (size_t t = 1; t < nt; ++t) pool.emplace_back(work);
  } catch (const std::system_error&) {
    // fewer threads than asked for: the ones that started (and this one) take the rest
  }
  work();
  for (std::thread& t : pool) t.join();
  for (int i = 0; i < n; ++i)
    if (status[i] != FTCC_OK) return status[i];
  return FTCC_OK;
}

ftcc_status ftcc_rdm2(ftcc_ctx* c, double* gamma) {
  if (!c || !gamma) return FTCC_ERR_INVALID_ARG;
  if (c->batch && c->batch->lambda_done && c->batch->adjoint_fp32)
    return fail(c, FTCC_ERR_UNSUPPORTED, "the two-particle density needs the FP64 adjoint (mixed_adjoint = 0)");
  if (!c->batch || !c->batch->lambda_done || !c->batch->s64 || c->batch->s64->fixed_bar.empty())
    return fail(c, FTCC_ERR_STATE, "the two-particle density needs ft_ccsd_adjoint first");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    Solver<double>& s = *B.s64;
    ftcc_ctx* h = B.home;
    CU(cudaSetDevice(h->device));
    const int N = B.N, no = B.no, nv = B.nv, z = c->member;
    const Inst& I = B.inst[z];
    const size_t N4 = static_cast<size_t>(N) * N * N * N;
    Buf g = h->get(N4 * sizeof(double));
    if (!g.p) throw Fail{FTCC_ERR_OOM, "allocation of the two-particle density failed"};
    CU(cudaMemsetAsync(g.p, 0, g.bytes, h->st));
    // dL/d<pq||rs> at a fixed reference: the adjoint of every thermal block
    // (integral times the slot factors of its letters) mapped back
    for (auto& kv : s.Vb) {
      auto it = s.fixed_bar.find(kv.second.p);
      if (it == s.fixed_bar.end()) continue;
      const std::string& pat = kv.first;
      const int* ix[4];
      const double* fx[4];
      int nn[4];
      long long total = 1;
      for (int k = 0; k < 4; ++k) {
        const bool ho = pat[k] == 'o';
        ix[k] = static_cast<const int*>(ho ? B.idxO.p : B.idxV.p);
        fx[k] = static_cast<const double*>(ho ? I.facO.p : I.facV.p);
        nn[k] = ho ? no : nv;
        total *= nn[k];
      }
      if (B.sparse)
        CU(launch_sp_eri_adjoint(static_cast<const double*>(it->second.p), static_cast<const int16_t*>(B.imp.p), N,
                                 fx[0], fx[1], fx[2], fx[3], static_cast<double*>(g.p), h->st));
      else
        CU(launch_eri_adjoint(static_cast<const double*>(it->second.p) + z * total, N, ix[0], fx[0], nn[0], ix[1],
                              fx[1], nn[1], ix[2], fx[2], nn[2], ix[3], fx[3], nn[3], static_cast<double*>(g.p),
                              h->st));
    }
    std::vector<double> raw(N4);
    CU(cudaMemcpyAsync(raw.data(), g.p, N4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    sync(h);
    h->put(g);
    // projection onto the symmetries of <pq||rs>: antisymmetric in (p, q)
    // and in (r, s), symmetric under (pq) <-> (rs)
    auto at = [&](int p, int q, int r, int t) { return raw[((static_cast<size_t>(p) * N + q) * N + r) * N + t]; };
    auto anti = [&](int p, int q, int r, int t) {
      return 0.25 * (at(p, q, r, t) - at(q, p, r, t) - at(p, q, t, r) + at(q, p, t, r));
    };
    for (int p = 0; p < N; ++p)
      for (int q = 0; q < N; ++q)
        for (int r = 0; r < N; ++r)
          for (int t = 0; t < N; ++t)
            gamma[((static_cast<size_t>(p) * N + q) * N + r) * N + t] = 0.5 * (anti(p, q, r, t) + anti(r, t, p, q));
    return FTCC_OK;
  });
}

ftcc_status ftcc_get_amplitudes(ftcc_ctx* c, double* s1, double* s2) {
  if (!c) return FTCC_ERR_INVALID_ARG;
  if (!c->batch) return fail(c, FTCC_ERR_STATE, "no prepared problem");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    ftcc_ctx* h = B.home;
    const long long g = B.ng, o = B.no, v = B.nv;
    const long long n1 = g * o * v, n2 = g * o * o * v * v;
    const long long z = c->member;
    if (B.sparse) {   // expand the compressed storage into the dense layouts
      Solver<double>& sv = *B.s64;
      Buf d1 = h->get(n1 * sizeof(double)), d2 = h->get(n2 * sizeof(double));
      if (!d1.p || !d2.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
      CU(launch_sp_expand(static_cast<const double*>(sv.t1.p), static_cast<const double*>(sv.t2.p),
                          static_cast<const int16_t*>(B.imp.p), B.N, B.ng, static_cast<double*>(d1.p),
                          static_cast<double*>(d2.p), h->st));
      if (s1) CU(cudaMemcpyAsync(s1, d1.p, n1 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      if (s2) CU(cudaMemcpyAsync(s2, d2.p, n2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      sync(h);
      h->put(d1);
      h->put(d2);
      return FTCC_OK;
    }
    Buf tmp = h->get(std::max(n1, n2) * sizeof(double));
    if (!tmp.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
    auto copy_out = [&](const void* base, long long n, double* dst) {
      if (B.active == 1)
        CU(launch_convert<float, double>(static_cast<const float*>(base) + z * n, static_cast<double*>(tmp.p), n, h->st));
      else
        CU(launch_convert<double, double>(static_cast<const double*>(base) + z * n, static_cast<double*>(tmp.p), n, h->st));
      CU(cudaMemcpyAsync(dst, tmp.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      sync(h);
    };
    if (s1) copy_out(B.active == 1 ? B.s32->t1.p : B.s64->t1.p, n1, s1);
    if (s2) copy_out(B.active == 1 ? B.s32->t2.p : B.s64->t2.p, n2, s2);
    h->put(tmp);
    return FTCC_OK;
  });
}

ftcc_status ftcc_eval_s(ftcc_ctx* c, int nx, int precision, const double* t1_dev, const double* t2_dev, double* s1_dev,
                        double* s2_dev) {
  if (!c || !t1_dev || !t2_dev || !s1_dev || !s2_dev) return FTCC_ERR_INVALID_ARG;
  if (!c->batch) return fail(c, FTCC_ERR_STATE, "ftcc_prepare first");
  if (c->batch->nz != 1) return fail(c, FTCC_ERR_STATE, "ftcc_eval_s works on a single prepared instance");
  if (nx < 1 || nx > c->batch->ng || precision < 0 || precision > 2)
    return fail(c, FTCC_ERR_INVALID_ARG, "bad nx or precision");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    const long long o = B.no, v = B.nv;
    const long long n1 = nx * o * v, n2 = nx * o * o * v * v;
    if (B.sparse) {
      // dense in and out: the inputs are projected onto the charge-conserving
      // elements (s1 diagonal, s2 with q_i + q_j = q_a + q_b), the outputs
      // expanded with zeros elsewhere
      // (TF32 / BF16X3: the FP32 block-sparse kernels of the mixed sweep, on
      // the rounded inputs, the outputs widened)
      const int nxc = precision == FTCC_PREC_FP64 ? make_solver<double>(B, GEMM_F64).nxc
                                                  : make_solver<float>(B, GEMM_BF16X3).nxc;
      if (nx > nxc) return fail(c, FTCC_ERR_INVALID_ARG, "nx exceeds the tau chunk");
      const long long N = B.N, n3 = N * N * N;
      Buf a = c->get(nx * N * 8), b = c->get(nx * n3 * 8), d = c->get(nx * N * 8), e = c->get(nx * n3 * 8);
      if (!a.p || !b.p || !d.p || !e.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
      const int16_t* imp = static_cast<const int16_t*>(B.imp.p);
      CU(cudaMemsetAsync(e.p, 0, nx * n3 * 8, c->st));   // the i = j / a = b elements of S2 are never written
      CU(launch_sp_compress(t1_dev, t2_dev, imp, B.N, nx, static_cast<double*>(a.p), static_cast<double*>(b.p), c->st));
      if (precision == FTCC_PREC_FP64) {
        Solver<double>& s = make_solver<double>(B, GEMM_F64);
        s.s_kernel(static_cast<double*>(a.p), static_cast<double*>(b.p), static_cast<double*>(d.p),
                   static_cast<double*>(e.p), nx);
      } else {
        Solver<float>& s = make_solver<float>(B, GEMM_BF16X3);
        Buf fa = c->get(nx * N * 4), fb = c->get(nx * n3 * 4), fd = c->get(nx * N * 4), fe = c->get(nx * n3 * 4);
        if (!fa.p || !fb.p || !fd.p || !fe.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
        CU(cudaMemsetAsync(fe.p, 0, nx * n3 * 4, c->st));
        CU(launch_convert<double, float>(static_cast<double*>(a.p), static_cast<float*>(fa.p), nx * N, c->st));
        CU(launch_convert<double, float>(static_cast<double*>(b.p), static_cast<float*>(fb.p), nx * n3, c->st));
        s.s_kernel(static_cast<float*>(fa.p), static_cast<float*>(fb.p), static_cast<float*>(fd.p),
                   static_cast<float*>(fe.p), nx);
        CU(launch_convert<float, double>(static_cast<float*>(fd.p), static_cast<double*>(d.p), nx * N, c->st));
        CU(launch_convert<float, double>(static_cast<float*>(fe.p), static_cast<double*>(e.p), nx * n3, c->st));
        sync(c);
        for (Buf* q : {&fa, &fb, &fd, &fe}) c->put(*q);
      }
      CU(launch_sp_expand(static_cast<double*>(d.p), static_cast<double*>(e.p), imp, B.N, nx, s1_dev, s2_dev, c->st));
      sync(c);
      for (Buf* q : {&a, &b, &d, &e}) c->put(*q);
    } else if (precision == FTCC_PREC_FP64) {
      Solver<double>& s = make_solver<double>(B, GEMM_F64);
      if (nx > s.nxc) return fail(c, FTCC_ERR_INVALID_ARG, "nx exceeds the tau chunk");
      s.s_kernel(t1_dev, t2_dev, s1_dev, s2_dev, nx);
    } else {
      if (!tma_available()) return fail(c, FTCC_ERR_UNSUPPORTED, "tensor-map encoder unavailable");
      Solver<float>& s = make_solver<float>(B, precision == FTCC_PREC_TF32 ? GEMM_TF32 : GEMM_BF16X3);
      if (nx > s.nxc) return fail(c, FTCC_ERR_INVALID_ARG, "nx exceeds the tau chunk");
      Buf a = c->get(n1 * 4), b = c->get(n2 * 4), d = c->get(n1 * 4), e = c->get(n2 * 4);
      if (!a.p || !b.p || !d.p || !e.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
      CU(launch_convert<double, float>(t1_dev, static_cast<float*>(a.p), n1, c->st));
      CU(launch_convert<double, float>(t2_dev, static_cast<float*>(b.p), n2, c->st));
      s.s_kernel(static_cast<float*>(a.p), static_cast<float*>(b.p), static_cast<float*>(d.p), static_cast<float*>(e.p), nx);
      CU(launch_convert<float, double>(static_cast<float*>(d.p), s1_dev, n1, c->st));
      CU(launch_convert<float, double>(static_cast<float*>(e.p), s2_dev, n2, c->st));
      sync(c);
      c->put(a);
      c->put(b);
      c->put(d);
      c->put(e);
    }
    sync(c);
    check_device_error(c);
    return FTCC_OK;
  });
}

ftcc_status ftcc_propagate(ftcc_ctx* c, const char* slots, const double* S_dev, double* s_dev) {
  if (!c || !slots || !S_dev || !s_dev) return FTCC_ERR_INVALID_ARG;
  if (!c->batch) return fail(c, FTCC_ERR_STATE, "ftcc_prepare first");
  if (c->batch->nz != 1) return fail(c, FTCC_ERR_STATE, "ftcc_propagate works on a single prepared instance");
  if (c->batch->sparse) return fail(c, FTCC_ERR_UNSUPPORTED, "block_sparse: dense layouts only");
  const int ns = static_cast<int>(strlen(slots));
  if (ns != 2 && ns != 4) return fail(c, FTCC_ERR_INVALID_ARG, "slots must be 'ia' or 'ijab'");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    PropArgs a = prop_args(B, ns);
    a.damping = 1.0;
    a.wE = nullptr;
    a.cE = 0.0;
    a.t1E = nullptr;
    a.nblocks = std::max(1, std::min(prop_blocks(), static_cast<int>((a.size + 127) / 128)));
    Buf part = c->get(static_cast<size_t>(a.nblocks) * (a.ng + 2) * sizeof(double));
    if (!part.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
    a.partials = static_cast<double*>(part.p);
    CU(cudaMemsetAsync(s_dev, 0, a.size * a.ng * sizeof(double), c->st));
    CU(launch_propagate<double>(S_dev, s_dev, a, c->st));
    sync(c);
    c->put(part);
    return FTCC_OK;
  });
}

ftcc_status ftcc_eval_s_vjp(ftcc_ctx* c, int nx, const double* t1_dev, const double* t2_dev, const double* w1_dev,
                            const double* w2_dev, double* t1bar_dev, double* t2bar_dev) {
  if (!c || !t1_dev || !t2_dev || !w1_dev || !w2_dev || !t1bar_dev || !t2bar_dev) return FTCC_ERR_INVALID_ARG;
  if (!c->batch) return fail(c, FTCC_ERR_STATE, "ftcc_prepare first");
  if (c->batch->nz != 1) return fail(c, FTCC_ERR_STATE, "works on a single prepared instance");
  if (nx < 1 || nx > c->batch->ng) return fail(c, FTCC_ERR_INVALID_ARG, "bad nx");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    Solver<double>& s = make_solver<double>(B, GEMM_F64);
    if (nx > s.nxc) return fail(c, FTCC_ERR_INVALID_ARG, "nx exceeds the tau chunk");
    if (B.sparse) {
      // dense in and out: inputs and cotangents projected onto the
      // charge-conserving elements, outputs expanded with zeros elsewhere
      const long long N = B.N, n3 = N * N * N;
      const int16_t* imp = static_cast<const int16_t*>(B.imp.p);
      Buf q[6];
      const long long sz[6] = {nx * N, nx * n3, nx * N, nx * n3, nx * N, nx * n3};
      for (int k = 0; k < 6; ++k) {
        q[k] = c->get(sz[k] * 8);
        if (!q[k].p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
      }
      double* d[6];
      for (int k = 0; k < 6; ++k) d[k] = static_cast<double*>(q[k].p);
      CU(launch_sp_compress(t1_dev, t2_dev, imp, B.N, nx, d[0], d[1], c->st));
      CU(launch_sp_compress(w1_dev, w2_dev, imp, B.N, nx, d[2], d[3], c->st));
      s.vjp(d[0], d[1], d[2], d[3], d[4], d[5], nx);
      CU(launch_sp_expand(d[4], d[5], imp, B.N, nx, t1bar_dev, t2bar_dev, c->st));
      sync(c);
      for (Buf& b : q) c->put(b);
      check_device_error(c);
      return FTCC_OK;
    }
    const long long n1 = nx * static_cast<long long>(B.no) * B.nv, n2 = n1 * B.no * B.nv;
    Buf a = c->get(n1 * 8), b = c->get(n2 * 8);
    if (!a.p || !b.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
    CU(cudaMemcpyAsync(a.p, w1_dev, n1 * 8, cudaMemcpyDeviceToDevice, c->st));
    CU(cudaMemcpyAsync(b.p, w2_dev, n2 * 8, cudaMemcpyDeviceToDevice, c->st));
    s.vjp(t1_dev, t2_dev, static_cast<double*>(a.p), static_cast<double*>(b.p), t1bar_dev, t2bar_dev, nx);
    sync(c);
    c->put(a);
    c->put(b);
    check_device_error(c);
    return FTCC_OK;
  });
}

ftcc_status ftcc_propagate_adjoint(ftcc_ctx* c, const char* slots, const double* m_dev, double* u_dev) {
  if (!c || !slots || !m_dev || !u_dev) return FTCC_ERR_INVALID_ARG;
  if (!c->batch) return fail(c, FTCC_ERR_STATE, "ftcc_prepare first");
  if (c->batch->sparse) return fail(c, FTCC_ERR_UNSUPPORTED, "block_sparse: dense layouts only");
  if (c->batch->nz != 1) return fail(c, FTCC_ERR_STATE, "works on a single prepared instance");
  const int ns = static_cast<int>(strlen(slots));
  if (ns != 2 && ns != 4) return fail(c, FTCC_ERR_INVALID_ARG, "slots must be 'ia' or 'ijab'");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    PropArgs a = prop_args(B, ns);
    a.nblocks = std::max(1, std::min(prop_blocks(), static_cast<int>((a.size + 127) / 128)));
    CU(launch_propagate_t(m_dev, u_dev, a, c->st));
    sync(c);
    return FTCC_OK;
  });
}

ftcc_status ftcc_get_lambda(ftcc_ctx* c, double* m1, double* m2) {
  if (!c) return FTCC_ERR_INVALID_ARG;
  if (!c->batch || !c->batch->lambda_done) return fail(c, FTCC_ERR_STATE, "run ft_ccsd_adjoint first");
  if (c->batch->sparse) return fail(c, FTCC_ERR_UNSUPPORTED, "block_sparse: dense layouts only");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    const long long n1 = static_cast<long long>(B.ng) * B.no * B.nv, n2 = n1 * B.no * B.nv;
    const long long z = c->member;
    if (B.adjoint_fp32) {
      std::vector<float> tmp;
      const std::pair<double*, long long> parts[2] = {{m1, n1}, {m2, n2}};
      for (int k = 0; k < 2; ++k) {
        if (!parts[k].first) continue;
        const long long n = parts[k].second;
        tmp.resize(n);
        CU(cudaMemcpyAsync(tmp.data(), static_cast<const float*>(k == 0 ? B.m1.p : B.m2.p) + z * n, n * 4,
                           cudaMemcpyDeviceToHost, B.home->st));
        sync(B.home);
        for (long long e = 0; e < n; ++e) parts[k].first[e] = tmp[e];
      }
      return FTCC_OK;
    }
    if (m1) CU(cudaMemcpyAsync(m1, static_cast<const double*>(B.m1.p) + z * n1, n1 * 8, cudaMemcpyDeviceToHost, B.home->st));
    if (m2) CU(cudaMemcpyAsync(m2, static_cast<const double*>(B.m2.p) + z * n2, n2 * 8, cudaMemcpyDeviceToHost, B.home->st));
    sync(B.home);
    return FTCC_OK;
  });
}

ftcc_status ftcc_profile(ftcc_ctx* c, int enable) {
  if (!c) return FTCC_ERR_INVALID_ARG;
  if (!c->batch) return fail(c, FTCC_ERR_STATE, "prepare or solve first");
  return run_guarded(c, [&]() -> ftcc_status {
    Batch& B = *c->batch;
    auto toggle = [&](auto* s) {
      if (!s) return;
      if (s->profiling != (enable != 0)) {
        if (s->gexec) cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
        if (s->graph) cudaGraphDestroy(s->graph);
        s->graph = nullptr;
        s->warm = false;   // the next iteration runs uncaptured, then a new graph with / without event nodes
      }
      s->profiling = enable != 0;
    };
    toggle(B.s32.get());
    toggle(B.s64.get());
    for (int k = 0; k < 8; ++k) {
      B.prof_ms[k] = B.prof_bytes[k] = B.prof_flops[k] = 0;
      B.prof_launches[k] = 0;
    }
    return FTCC_OK;
  });
}

int ftcc_profile_read(ftcc_ctx* c, ftcc_kernel_stats* out, int max) {
  if (!c || !c->batch || !out || max < 1) return 0;
  Batch& B = *c->batch;
  int n = 0;
  for (int k = 0; k < kNumCls && n < max; ++k) {
    if (B.prof_launches[k] == 0) continue;
    ftcc_kernel_stats& r = out[n++];
    memset(&r, 0, sizeof(r));
    strncpy(r.name, kClsName[k], sizeof(r.name) - 1);
    r.launches = B.prof_launches[k];
    r.ms = B.prof_ms[k];
    r.bytes = B.prof_bytes[k];
    r.flops = B.prof_flops[k];
  }
  return n;
}

ftcc_status ftcc_gemm(ftcc_ctx* c, int precision, int batch, int M, int N, int K, double alpha, const void* A,
                      long long lda, long long sa, const void* B, long long ldb, long long sb, void* C, long long ldc,
                      long long sc) {
  if (!c || !A || !B || !C || batch < 1 || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N || sa < 0 || sb < 0 ||
      sc < 0 || precision < 0 || precision > 2)
    return FTCC_ERR_INVALID_ARG;
  if (precision != FTCC_PREC_FP64 &&
      ((lda % 4) || (ldb % 4) || (sa % 4) || (sb % 4) || (reinterpret_cast<uintptr_t>(A) & 15) ||
       (reinterpret_cast<uintptr_t>(B) & 15)))
    return fail(c, FTCC_ERR_INVALID_ARG, "tensor-core operands need 16-byte aligned rows");
  return run_guarded(c, [&]() -> ftcc_status {
    GemmArgs g{};
    g.batch = batch;
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = A;
    g.lda = lda;
    g.sa = sa;
    g.B = B;
    g.ldb = ldb;
    g.sb = sb;
    g.C = C;
    g.ldc = ldc;
    g.sc = sc;
    g.alpha = alpha;
    g.beta = 0.0;
    // split-K partials when the output alone cannot fill the SMs
    const size_t wbytes = std::min<size_t>(64u << 20, static_cast<size_t>(batch) * M * N * 8 * 32);
    Buf w = c->get(wbytes);
    g.work = w.p;
    g.work_bytes = w.bytes;
    struct Release {
      ftcc_ctx* c;
      Buf& b;
      ~Release() {
        cudaStreamSynchronize(c->st);
        c->put(b);
      }
    } release{c, w};
    if (precision == FTCC_PREC_FP64) {
      CU(gemm_f64(g, c->st));
    } else if (precision == FTCC_PREC_TF32) {
      if (!tma_available()) return fail(c, FTCC_ERR_UNSUPPORTED, "tensor-map encoder unavailable");
      CU(gemm_tc(GEMM_TF32, g, c->dev_err, c->st));
    } else {
      // split FP32 operands into bf16 hi / lo in scratch, then three tensor-core products
      if (!tma_available()) return fail(c, FTCC_ERR_UNSUPPORTED, "tensor-map encoder unavailable");
      const long long kp = (K + 63) / 64 * 64;
      const long long ra = static_cast<long long>(batch) * M, rb = static_cast<long long>(batch) * N;
      Buf ah = c->get(ra * kp * 2), al = c->get(ra * kp * 2), bh = c->get(rb * kp * 2), bl = c->get(rb * kp * 2);
      if (!ah.p || !al.p || !bh.p || !bl.p) throw Fail{FTCC_ERR_OOM, "allocation failed"};
      PackDesc d{};
      d.nr = 2;
      d.nc = 1;
      d.rdim[0] = batch;
      d.rst[0] = sa;
      d.rdim[1] = M;
      d.rst[1] = lda;
      d.cdim[0] = K;
      d.cst[0] = 1;
      d.rows = ra;
      d.creal = K;
      d.cpad = kp;
      CU(launch_pack_bf16x2(static_cast<const float*>(A), ah.p, al.p, d, c->st));
      d.rdim[0] = batch;
      d.rst[0] = sb;
      d.rdim[1] = N;
      d.rst[1] = ldb;
      d.rows = rb;
      CU(launch_pack_bf16x2(static_cast<const float*>(B), bh.p, bl.p, d, c->st));
      g.A = ah.p;
      g.A2 = al.p;
      g.B = bh.p;
      g.B2 = bl.p;
      g.lda = kp;   // K stays the true length: columns K..kp are never read
      g.ldb = kp;
      g.sa = sa > 0 ? M * kp : 0;
      g.sb = sb > 0 ? N * kp : 0;
      CU(gemm_tc(GEMM_BF16X3, g, c->dev_err, c->st));
      sync(c);
      c->put(ah);
      c->put(al);
      c->put(bh);
      c->put(bl);
    }
    sync(c);
    check_device_error(c);
    return FTCC_OK;
  });
}

ftcc_status ftcc_inject_device_error(ftcc_ctx* c, int code) {
  if (!c || code <= 0) return FTCC_ERR_INVALID_ARG;
  return run_guarded(c, [&] {
    CU(cudaSetDevice(c->device));
    CU(cudaMemcpyAsync(c->dev_err, &code, sizeof(int), cudaMemcpyHostToDevice, c->st));
    sync(c);
    return FTCC_OK;
  });
}

int ftcc_device_error(ftcc_ctx* c) {
  if (!c) return -1;
  int e = 0;
  if (cudaMemcpyAsync(&e, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess) return -1;
  cudaStreamSynchronize(c->st);
  cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->st);
  cudaStreamSynchronize(c->st);
  return e;
}

}  // extern "C"
