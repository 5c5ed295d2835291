// Internal declarations of libftcc (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ftcc.h"

namespace ftcc {

// Precision of the GEMM engine.
enum GemmKind { GEMM_F64 = 0, GEMM_TF32 = 1, GEMM_BF16X3 = 2 };

// Device error codes written by bounded waits (0 = no error).
enum DeviceError { DEVERR_NONE = 0, DEVERR_TMA_TIMEOUT = 1, DEVERR_MMA_TIMEOUT = 2, DEVERR_EPI_TIMEOUT = 3 };

// Allocation through the context's allocator.
struct Alloc {
  ftcc_allocator a;
  bool custom = false;
  void* get(size_t bytes);
  void put(void* p);
};

// A device buffer owned by the context.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

// ---- GEMM engine (gemm_tc.cu, gemm_f64.cu) --------------------------------
// C[b][m][n] = alpha * sum_k A[b][m][k] * B[b][n][k] + beta * C[b][m][n]
// A, B row-major with K contiguous.  Batch strides in elements (0 = shared).
struct GemmArgs {
  int batch, M, N, K;
  void* work; size_t work_bytes;      // split-K partials for the SIMT kernels (may be null)
  const void* A; long long lda, sa;
  const void* B; long long ldb, sb;
  const void* A2; const void* B2;     // low halves for BF16X3 (bf16 arrays)
  void* C; long long ldc, sc;
  double alpha, beta;
  int trans;                          // 1: C stored transposed, element (m, n) at C[b*sc + n*ldc + m]
  int bn, split;                      // tensor-core tile width and K splits (0: the built-in choice)
};
// Tensor-core GEMM (tcgen05 + TMA).  kind TF32: A, B, C float.  kind BF16X3:
// A, A2, B, B2 __nv_bfloat16 (hi, lo), C float.  Returns cudaSuccess or an error.
cudaError_t gemm_tc(int kind, const GemmArgs& g, int* dev_err, cudaStream_t st);
// FP64 SIMT GEMM.
cudaError_t gemm_f64(const GemmArgs& g, cudaStream_t st);
// FP32 SIMT GEMM (used where a tensor-core tile would be mostly padding).
cudaError_t gemm_f32(const GemmArgs& g, cudaStream_t st);
// Row-per-thread kernels for N <= 32 and K <= 32 (full FP32 / FP64 arithmetic).
bool gemm_skinny_fits(const GemmArgs& g);
cudaError_t gemm_skinny_f32(const GemmArgs& g, cudaStream_t st);
cudaError_t gemm_skinny_f64(const GemmArgs& g, cudaStream_t st);
bool tma_available();

}  // namespace ftcc

namespace ftcc {

constexpr int kMaxL = 6;   // letters per tensor (x plus up to four orbital slots)

// Unsigned 32-bit division by an invariant d >= 1 as a multiply-high and a
// shift: with s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> s for every n < 2^32 (sum taken in 64 bits).
struct FastDiv {
  uint32_t d, m, s;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.s = 0;
  while ((1ull << f.s) < d) ++f.s;
  f.m = static_cast<uint32_t>((((1ull << 32) * ((1ull << f.s) - d)) / d) + 1);
  return f;
}

// Gather a strided source into a row-major [rows][cpad] operand.  The
// padding columns creal..cpad are left unwritten: every GEMM reads only the
// first creal columns (the tensor maps have K = creal and fill the rest of
// a box with zeros).  Row index = mixed radix over rdim (last fastest), column
// index over cdim; source offset = sum coord * stride.
struct PackDesc {
  int nr, nc;
  long long rdim[kMaxL], rst[kMaxL], cdim[kMaxL], cst[kMaxL];
  long long rows, creal, cpad;
};
// dst[e] = beta * dst[e] + alpha * sum_p sign_p * src[off_p(e)] where the
// terms p run over the antisymmetriser: identity, swap(s0a, s0b),
// swap(s1a, s1b), both swaps (signs +, -, -, +); nswap = 0, 1, 2.  A source
// stride of 0 broadcasts along that letter.  Both launchers run the tiled
// permute kernel (shared-memory tiles, coalesced reads and writes; each term
// read in its own letter order).
// Unordered pairs (p < q) of antisymmetric tensors: pack [b][P][Q] from a
// strided four-index tensor (optionally antisymmetrising the first pair), and
// add the dense antisymmetric tensor of a packed [b][P_ij][P_ab] one.
template <class T>
cudaError_t launch_pair_pack(const T* src, T* dst, long long nb, long long sb, const int2* pairs1, long long np1,
                             const int2* pairs2, long long np2, long long s0, long long s1, long long s2, long long s3,
                             int anti, double coef, cudaStream_t st);
template <class T>
cudaError_t launch_pair_unpack_add(T* R, const T* L, long long nb, int no, int nv, double coef, cudaStream_t st);
// Contiguous-block copy (see launch_block_copy): the destination's leading
// letters (dim, outermost first) with the source strides of those letters (0
// where the source lacks one).
struct BlockCopyDesc {
  int nouter;
  long long dim[kMaxL], sst[kMaxL];
};
template <class T>
cudaError_t launch_block_copy(T* dst, const T* src, long long B, const BlockCopyDesc& d, double alpha, double beta,
                              cudaStream_t st);
// hi / lo bf16 halves of rows already in GEMM order (row strides sld, ld).
cudaError_t launch_split_rows(const float* src, long long sld, void* hi, void* lo, long long ld, long long rows,
                              long long K, cudaStream_t st);
struct ScatDesc {
  int nd;
  long long dim[kMaxL], sst[kMaxL];
  int nswap;
  int sw[2][2];
  long long total;
};

// dst[zx][i][j][a][b] (dense) = sum_s coef_s P(ij)P(ab) X_s + V(ab,ij): element
// (zx,i,j,a,b) of source s at p + zx*sx + i*si + j*sj + a*sa + b*sb; V at
// vp + z*vz + a*va + b*vb + i*vi + j*vj with z = zx / nx (vp may be null).
// Each unordered pair {i,j} and pair of 32-wide a/b tiles is evaluated once;
// the result is exactly antisymmetric.  One or two sources.
struct AntiSrc {
  const void* p;
  long long sx, si, sj, sa, sb;
  double coef;
};
struct Anti4Desc {
  int nzx, nx, no, nv, nsrc;
  int ta;                      // tile edge (set by the launcher)
  AntiSrc src[2];
  const void* vp;
  long long vz, va, vb, vi, vj;
};
template <class T> cudaError_t launch_antisym4(T* dst, const Anti4Desc& d, cudaStream_t st);
template <class T> cudaError_t launch_pack(const T* src, T* dst, const PackDesc& d, cudaStream_t st);
cudaError_t launch_pack_bf16x2(const float* src, void* hi, void* lo, const PackDesc& d, cudaStream_t st);
template <class T> cudaError_t launch_scatter(const T* src, T* dst, const ScatDesc& d, double alpha,
                                              double beta, cudaStream_t st);
// tt = t2 + c_tt * (t1 t1 antisymmetrised), ta likewise with c_ta, and
// X_ijab = 1/2 t2_ijab + t1_ia t1_jb (any output may be null), one read of t2
template <class T> cudaError_t launch_tau(const T* t1, const T* t2, T* tt, T* ta, T* X, double c_tt, double c_ta,
                                          int nx, int no, int nv, cudaStream_t st);
template <class Ts, class Td> cudaError_t launch_convert(const Ts* s, Td* d, long long n, cudaStream_t st);

// ---- physics (App. A) ----
cudaError_t launch_hubbard(double* h, double* eri, double* eps, int L, double t, double U, cudaStream_t st);
cudaError_t launch_ueg(double* h, double* eri, double* eps, const int* nvec, int M, int nocc, double vol,
                       double kunit, cudaStream_t st);
// n, nbar, f = h + sum_r n_r <pr||qr>, fbar = f - diag(eps)
cudaError_t launch_reference(const double* h, const double* eri, const double* eps, int N, double beta,
                             double mu, double* n, double* nbar, double* f, double* fbar, double* scal,
                             cudaStream_t st);
// em[p] = exp(-eps_p h), ep[p] = exp(eps_p h)
cudaError_t launch_prop_tables(const double* eps, int N, double h, double* em, double* ep, cudaStream_t st);
// thermal block: out[p0][p1][p2][p3] = eri[...] * fac(slot0) * ... with per-slot index lists
cudaError_t launch_eri_adjoint(const double* bar, int N, const int* idx0, const double* fac0, int n0, const int* idx1,
                              const double* fac1, int n1, const int* idx2, const double* fac2, int n2,
                              const int* idx3, const double* fac3, int n3, double* gamma, cudaStream_t st);
template <class T> cudaError_t launch_thermal_eri(const double* eri, int N, const int* idx0, const double* fac0,
                                                  int n0, const int* idx1, const double* fac1, int n1,
                                                  const int* idx2, const double* fac2, int n2, const int* idx3,
                                                  const double* fac3, int n3, T* out, cudaStream_t st);
template <class T> cudaError_t launch_thermal_fock(const double* fbar, int N, const int* idx0, const double* fac0,
                                                   int n0, const int* idx1, const double* fac1, int n1, T* out,
                                                   cudaStream_t st);
// Propagation + fused energy (see kernels.cu).
struct PropArgs {
  int ng, nslot;                 // nslot 2 (singles) or 4 (doubles)
  long long size;                // elements per tau slice of one instance (< 2^31)
  int no, nv;
  int nz, N;                     // instances (blockIdx.y), spin orbitals
  FastDiv fo, fv;                // filled by the launcher
  const int* idxO; const int* idxV;
  const double* em; const double* ep;   // [nz][N]
  const double* hz;              // [nz] grid steps
  const int* live;               // [nz] 0 = instance frozen (diverged), or null
  double damping;
  const double* wE;              // [nz][size] energy weights (f_ia or <ij||ab>) or null
  double cE;                     // coefficient of wE * s
  const void* t1E;               // [nz][ng][o][v] new singles, same type as t, or null
  double* partials;              // [nz][ng + 2][nblocks]
  int nblocks;                   // blocks per instance
  // tau points [y0, y1) of this launch; S holds s_ng points per instance
  // starting at y0.  chain ([nz][5][size], same type as t) carries the
  // recurrence between launches; it may be null only for y0 = 0, y1 = ng.
  int y0, y1, s_ng;
  void* chain;
  // block-sparse storage (null: dense): doubles are [i][j][a] with b =
  // imp[i][j][a] (no = nv = N, holes skipped), singles the diagonal [i]
  const int16_t* imp;
  // with imp, propagation of the doubles only: the canonical elements
  // (i < j, a < b) of the antisymmetric s2; each is propagated once and
  // written to its four orientations with their signs (the energy and the
  // maxima count it for all four)
  const int* canon;
  long long ncanon;
  int arith64;                   // FP32 storage: 0 = FP32 recurrence and energy sums, 1 = FP32
                                 // recurrence with FP64 energy sums, 2 = FP64 for both
};
template <class T> cudaError_t launch_propagate(const T* S, T* t, const PropArgs& a, cudaStream_t st);
// Site-basis Hubbard ring with the Neel or UHF reference (references.cu):
// h [N*N], <pq||rs> [N^4], eps [N] on the host; false with err on failure.
bool hubbard_site_reference(int L, double t, double U, int reference, std::vector<double>& h,
                            std::vector<double>& eri, std::vector<double>& eps, std::string& err);
int prop_blocks();
// Per instance z, sum the partials of the singles and doubles passes; row
// state[z][.]: 0 <- Omega_CC, 1 <- |dOmega_CC|, 2 <- max|ds|/max(1, max|s|),
// 3 <- previous Omega_CC, 8 + y <- E(tau_y).  hz holds [nz] steps then [nz] betas.
// ---- differential form (Eq. smud) marched by explicit RK steps (rk.cu) ----
// up to four stage derivatives K_j with their coefficients
template <class T>
struct RkTerms {
  int n;
  T c[4];
  const T* K[4];
};
// out[z][mu] = base[z][mu] + hz[z] sum_j c_j K_j[z][mu] (K_j dense [nz][n])
template <class T>
cudaError_t launch_rk_combine(T* out, long long out_zstride, const T* base, long long base_zstride,
                              const RkTerms<T>& k, const double* hz, long long n, int nz, cudaStream_t st);
// K = -(Delta Y + S) for the singles (nslot 2) or doubles (nslot 4) of nz instances
template <class T>
cudaError_t launch_rk_deriv(T* K, const T* Y, const T* S, const double* eps, const int* idxO, const int* idxV, int N,
                            int no, int nv, int nslot, int nz, cudaStream_t st);
// per-block energy partials of every tau point (Eq. E) in the layout launch_reduce folds
template <class T>
cudaError_t launch_rk_energy(const T* t1, const T* t2, const double* F64, const double* V64, int ng, int no, int nv,
                             int nz, int nb1, int nb2, double* part1, double* part2, cudaStream_t st);
cudaError_t launch_reduce(const double* p1, int nb1, const double* p2, int nb2, int ng, int nz, const double* hz,
                          const int* live, double* state, cudaStream_t st);
double simpson_weight_host(int y, int ng);

// ---- adjoint ----
// u[z][x][mu] = sum_y G[y,x] exp(-Delta (tau_y - tau_x)) m[z][y][mu] (transpose of the propagation)
template <class T> cudaError_t launch_propagate_t(const T* m, T* u, const PropArgs& a, cudaStream_t st);
// m_new = -c[z][x] * base' - tbar with base' = cbase * base[z][mu] (cbase != 0, tau-independent base)
// or base[z][x][mu] (cbase == 0); partials [nblocks][2] = max|m_new - m_old|, max|m_new|.  With a
// list, only the positions mu of the list (block-sparse valid positions; the rest stays zero)
template <class T, class BT>
cudaError_t launch_lambda_combine(const BT* base, const T* tbar, T* mnew, const T* mold, long long size, int ng, int nz,
                                  const double* cz, double cbase, double* partials, int nblocks, cudaStream_t st,
                                  const int* list = nullptr, int nlist = 0);

// ---- response (App. B) ----
// Do[z][q] / Dv[z][q] += sum A*I over elements with a hole-like / particle-like
// slot at position q; cls bit k set = slot k particle-like.  dims[nslot].
template <class T>
cudaError_t launch_slot_sums(const T* I, const T* A, int nslot, const int* dims, int cls, int no, int nv, int nz,
                             double* Do, double* Dv, cudaStream_t st);
template <class T>
cudaError_t launch_fbar_scatter(const T* A, int n0, int n1, const int* i0, const double* f0, long long f0z,
                                const int* i1, const double* f1, long long f1z, int N, int nz, double* Fb,
                                cudaStream_t st);
cudaError_t launch_fock_n(const double* Fb, const double* eri, int N, double* Gn, cudaStream_t st);
template <class T>
cudaError_t launch_prop_response(const T* S, const T* m, const double* epsz, const PropArgs& a, double* Ee, double* Eb,
                                 cudaStream_t st);

// ---- momentum/spin block-sparse S kernel (sparse.cu), FP64 ----
// Four-index tensors are N^3 arrays [p0][p1][p2] with q_p0 + q_p1 = q_p2 + q_p3
// and p3 implied; imp[a][b][c] (int16, N^3) = the orbital of charge
// q_a + q_b - q_c or -1.  Two-index tensors are their diagonals [p].
template <class T>
struct SpBlocksT {   // thermal integral blocks <pq||rs> of each hole / particle class, N^3 each
  const T *oovv, *ovvv, *ooov, *oooo, *vvvv, *ovvo, *oovo, *ovov, *vvoo, *vvvo, *ovoo;
};
using SpBlocks = SpBlocksT<double>;
template <class T>
struct SpVecArgsT {
  const T *t1, *t2;
  const T *fov, *foo, *fvv, *fvo;   // diagonals of the thermal Fock blocks
  const T *Voovv, *Vovvv, *Vooov, *Vovov, *Voovo;
  const int16_t* imp;
  // per orbital p, the (m, q) = m n + q with a valid position (m, q, p) (l1)
  // and (p, m, q) (l2); offsets [n + 1]
  const int *l1, *off1, *l2, *off2;
  int n;
  T *Fme, *Fae, *Fmi, *S1, *Ft, *Ft2;   // [nx][n] each
};
// Products of the blocks of one pair-charge sector (see sparse.cu).
template <class T>
struct SecGemmArgsT {
  const T* A;
  long long ax;          // slice stride of A
  const T* B;
  long long bx;          // slice stride of B (0: fixed)
  T* C;
  long long cx;
  double alpha;
  int n;
  int swapB;
  long long s0, s1, s2, s3;   // output position = p_r s0 + q_r s1 + p_c s2 + q_c s3
  const int2* ent;       // ordered pairs of every sector, sector by sector
  const int* kl;         // summed-index list of every sector
  const int4* sec;       // (entry offset, rows, K offset, K count)
  const int4* work;      // (sector, row tile start, column tile start, 0)
  // optional second product over the same rows and K list: C += alpha (A B^T + A2 B2^T)
  const T* A2;
  const T* B2;
  // anti4: rows (i, j), columns (a, b); the value is added to C[i][j][a],
  // C[j][i][a] (-), C[i][j][b] (-), C[j][i][b] (N^3 storage, the fourth index
  // implied), i.e. to all four orientations of an antisymmetric result
  int anti4;
  // store (without anti4): C[q] = value, for an output that no other term
  // touches (every position written exactly once), instead of C[q] += value
  int store;
};
using SecGemmArgs = SecGemmArgsT<double>;
// Transposed sector products (see sparse.cu): D[orow(e_o)][k] += alpha
// sum_{e_s} G[gpos(e_o, e_s)] A[srow(e_s)][k]; dx = 0: D fixed, the kernel
// sums the nx slices of G and A.
struct SecTnArgs {
  double* D;
  long long dx;
  const double* G;
  long long gx;
  const double* A;
  long long ax;
  double alpha;
  int n, nx;
  int swapD, swapA;
  long long g0, g1, g2, g3;   // gpos = p_o g0 + q_o g1 + p_s g2 + q_s g3
  const int2* ent;
  const int* kl;
  const int4* sec;
  const int4* work;
  // unordered sectors (pairs p < q): antiA reads A antisymmetrised in its
  // row pair, (A[p q] - A[q p]) / 2; anti4 writes each output (p_o q_o, k l)
  // to its four orientations with signs +, -, -, + (l the partner of k)
  int antiA, anti4;
};
// Forward values and cotangents of the block-sparse S-kernel transpose ([nx][N^3] / [nx][N]).
struct SpVjpArgs {
  const double *t1, *t2;
  const double *Ft, *Ft2, *Fme, *Fae, *Fmi;          // forward vectors
  const double *S1b;                                 // cotangent of S1
  const double *Rb, *w1b, *wabb, *wrb, *tab, *tpb, *trb, *xpb;
  SpBlocks V;
  const int16_t* imp;
  const int* list;                                   // the valid N^3 positions
  int nlist;
  const int *l1, *off1, *l2, *off2;                  // per orbital p: valid (m, q) of (m, q, p) / (p, m, q)
  int n;
  double *Ftb, *Ft2b, *Faeb, *Fmib, *Fmeb;           // vector cotangents (written)
  double *t1b, *t2b;                                 // outputs (the holes of t2b must be zero: not written)
};
cudaError_t launch_sp_s2_t(const double* S2b, const int16_t* imp, const int* list, int nlist, int n, int nx,
                           double* Rb, cudaStream_t st);
cudaError_t launch_sector_tn(const SecTnArgs& g, int nwork, cudaStream_t st);
cudaError_t launch_sector_tn_small(const SecTnArgs& g, int nwork, cudaStream_t st);   // sectors of <= 16 pairs
cudaError_t launch_sp_vjp_vectors(const SpVjpArgs& v, int nx, cudaStream_t st);
cudaError_t launch_sp_t2bar(const SpVjpArgs& v, int nx, cudaStream_t st);
// Vbar[11] in SpBlocks order (null entries skipped), fbar[4] = ov, vv, oo, vo (null skipped); cz may be null
cudaError_t launch_sp_fixed_bar(const SpVjpArgs& v, const double* S2b, const double* cz, double* const* Vbar,
                                double* const* fbar, int nx, cudaStream_t st);
cudaError_t launch_sp_swap12_add(const double* in, int n, double* out, cudaStream_t st);   // out[a][b][c] += in[a][c][b]
cudaError_t launch_sp_eri_adjoint(const double* bar, const int16_t* imp, int n, const double* f0, const double* f1,
                                  const double* f2, const double* f3, double* gamma, cudaStream_t st);
cudaError_t launch_sp_energy_bar(const double* t1, const double* t2, const double* cz, const int16_t* imp, int n,
                                 int ng, double* Voovvb, double* fovb, cudaStream_t st);
// Do[q] / Dv[q] += sum of I * Ib over the elements with orbital q in a hole-like / particle-like
// slot (bit k of cls set = slot k particle-like; slot 3 is the implied one)
cudaError_t launch_sp_slot_sums(const double* I, const double* Ib, const int16_t* imp, int n, int cls, double* Do,
                                double* Dv, cudaStream_t st);
// out[x][m] = fov[m] + sum_n s1[x][n] <mn||mn>  (F_me, and dE/ds1 of Eq. E)
cudaError_t launch_sp_fme(const double* t1, const double* fov, const double* Voovv, int n, int nx, double* out,
                          cudaStream_t st);
// skip_tau: leave ta, tp to launch_sp_canon (the unordered-pair products read only their canonical elements)
// list (may be null): with skip_tau, the positions whose (p0, p2, p1) is valid (tr, xp only)
template <class T>
cudaError_t launch_sp_amp(const T* t1, const T* t2, const int16_t* imp, int n, int nx, T* ta, T* tp, T* tr, T* xp,
                          int skip_tau, const int* list, int nlist, cudaStream_t st);
// ta, tp and the antisymmetrised W'_mnij, W'_abef at the canonical positions (p0 < p1, p2 < p3) only
template <class T>
cudaError_t launch_sp_canon(const T* t1, const T* t2, const SpBlocksT<T>& V, const int16_t* imp, const int* canon,
                            int ncanon, int n, int nx, T* ta, T* tp, T* w1, T* wab, cudaStream_t st);
template <class T> cudaError_t launch_sp_vectors(const SpVecArgsT<T>& v, int nx, cudaStream_t st);
// anti != 0: only W_mbej (the antisymmetrised W'_mnij, W'_abef of the
// unordered-pair ladders come from launch_sp_canon)
// list (may be null): with anti, the positions (p0, p1, p2) whose (p1, p2, p0) is valid (W_mbej only)
template <class T>
cudaError_t launch_sp_wbase(const T* t1, const SpBlocksT<T>& V, const int16_t* imp, int n, int nx, T* w1, T* wab,
                            T* wr, int anti, const int* list, int nlist, cudaStream_t st);
// R over the valid positions (list) only
template <class T>
cudaError_t launch_sp_rinit(const T* t1, const T* t2, const T* Ft, const T* Ft2, const SpBlocksT<T>& V,
                            const int16_t* imp, const int* list, int nlist, int n, int nx, T* R, cudaStream_t st);
// S2 from its canonical elements, written to their four orientations; R is
// [i][j][a] (b implied), Xr the ring term [i][a][b] (j implied) or null, Lc
// a term given at the canonical elements only (added once) or null
template <class T>
cudaError_t launch_sp_s2(const T* R, const T* Xr, const T* Lc, const T* Vvvoo, const int16_t* imp, const int* canon,
                         int ncanon, int n, int nx, T* S2, cudaStream_t st);
template <class T> cudaError_t launch_sector_gemm(const SecGemmArgsT<T>& g, int nwork, int nx, cudaStream_t st);
// the same products for work items of sectors of at most 16 pairs (16 x 16 tiles, 64 threads)
template <class T>
cudaError_t launch_sector_gemm_small(const SecGemmArgsT<T>& g, int nwork, int nx, cudaStream_t st);
int sector_tile();
template <class T>
cudaError_t launch_sp_thermal_eri(const double* eri, const int16_t* imp, int n, const double* f0, const double* f1,
                                  const double* f2, const double* f3, T* out, cudaStream_t st);
template <class T> cudaError_t launch_sp_swap12(const T* in, int n, T* out, cudaStream_t st);   // out[a][b][c] = in[a][c][b]
template <class T>
cudaError_t launch_sp_thermal_fock(const double* fbar, int n, const double* f0, const double* f1, T* out,
                                   cudaStream_t st);
cudaError_t launch_sp_compress(const double* d1, const double* d2, const int16_t* imp, int n, int nx, double* s1,
                               double* s2, cudaStream_t st);
cudaError_t launch_sp_expand(const double* s1, const double* s2, const int16_t* imp, int n, int nx, double* d1,
                             double* d2, cudaStream_t st);

}  // namespace ftcc
