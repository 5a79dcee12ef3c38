// Internal declarations of the shbim library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "shbim.h"

namespace shbim {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 0.07957747154594766788;   // 1/(4 pi)
constexpr double kSqrt2 = 1.41421356237309504880;

inline int ncoef(int p) { return (p + 1) * (p + 1); }
inline int ntri(int p) { return (p + 1) * (p + 2) / 2; }
inline int nlat(int q) { return q + 1; }
inline int nlon(int q) { return 2 * q + 2; }
inline int npts(int q) { return (q + 1) * (2 * q + 2); }

// Number of Laplace / Stokes weight components in the singular self rows.
constexpr int kNumLap = 2;        // 0: double layer (target normal), 1: single layer
constexpr int kNumSto = 12;       // 0..5 Stokeslet xx,xy,xz,yy,yz,zz ; 6..11 stresslet (same order)
constexpr double kNearFactor = 6.0;  // near zone: 6 source-grid spacings

// Legendre tables per latitude (kinds of the synthesis). "phi-type" tables multiply the
// sin/cos-swapped Fourier sum (a phi derivative); the others the plain one.
constexpr int kNumTab = 7;
//   0 Pbar            1 dPbar/dtheta        2 m Pbar / sin (phi-type)
//   3 d2Pbar/dtheta2  4 m dPbar/dtheta (phi-type)   5 -m^2 Pbar   6 m Pbar (phi-type)
// so that kinds 0,1,2 give f, f_theta, f_phi / sin and kinds 0,1,6,3,4,5 give f, f_theta,
// f_phi, f_theta_theta, f_theta_phi, f_phi_phi.
constexpr int kPhiTypeMask = (1 << 2) | (1 << 4) | (1 << 6);

// Transform tables of one (p, grid degree q) pair, device memory.
struct GridTables {
  int p = 0, q = 0;
  double* alf = nullptr;     // [q+1][kNumTab][ntri(p)] m-major (see kNumTab)
  double* omega = nullptr;   // [q+1] regular weight (pi/(q+1)) w_j^G
  double* mu = nullptr;      // [q+1] modified weight omega_j 2 sin(theta_j/2) sum_{n<=q} P_n(t_j)
  double* trig = nullptr;    // [2][2q+2] cos, sin of 2 pi k / (2q+2)
  double* theta = nullptr;   // [q+1]
  float* alf32 = nullptr;    // [q+1][ntri(p)] Pbar in FP32 (FP32 synthesis of strengths), or null
  float* trig32 = nullptr;   // [2][2q+2] in FP32
};

struct DegreeTables {
  int p = 0;
  GridTables base;           // q = p
  GridTables up;             // q = 2p+1
  GridTables fine;           // q = 4(2p+2) - 1: nearly-singular sums
  double* dq = nullptr;      // rotation matrix blocks of Rx(pi/2), sum_n (2n+1)^2 doubles
  std::vector<int> dq_off;   // host copy of block offsets (n -> offset)
  int* dq_off_dev = nullptr;
  // double-float copies (hi, lo) for the double-float singular-row build (singular_df.cu)
  float2* up_alf_df = nullptr;   // [2p+2 latitudes][3][ntri(p)]: Pbar, dPbar/dtheta, m Pbar/sin
  float2* up_trig_df = nullptr;  // [2][4p+4]: cos, sin of 2 pi k / (4p+4)
  float2* dq_df = nullptr;       // as dq
  // nonzero pattern of the Dq blocks (about a quarter of the entries; parity structure of the
  // quarter turn): per row and per column of every block, the nonzero entries as an arithmetic
  // progression (start, count, step) of column (row) indices, indexed like the coefficients
  int4* dq_rows = nullptr;       // [(p+1)^2]
  int4* dq_cols = nullptr;       // [(p+1)^2]
  float2* cs_theta_df = nullptr; // [p+1 base latitudes][2][p+1]: cos(m theta_j), sin(m theta_j)
  float2* cs_phi_df = nullptr;   // [2p+2 base longitudes][2][p+1]: cos(m phi_k), sin(m phi_k)
  // digit planes of the up-grid DFT table for the tensor-core Fourier analysis (dft_tc.cu):
  // [n tile][K step][digit][80 outputs x 16 longitudes, K-major canonical layout], bfloat16
  uint16_t* dft_digits = nullptr;
  int dft_ntiles = 0, dft_ksteps = 0;
  // digit planes of Dq_n^T Dz(-+theta_j) Dq_n per base-grid latitude for the tensor-core rotations
  // (rot_tc.cu), p <= 39: [2][p+1][p+1][K step][digit][Np x 16], with per-(direction, latitude,
  // degree) offsets in 16-byte units
  uint16_t* rot_digits = nullptr;
  int* rot_toff = nullptr;
  signed char* rot_exp = nullptr;   // [2][p+1][(p+1)^2] row exponents of the tables
  // digit planes of Pbar_n^m at the degree 2p+1 grid latitudes for the tensor-core Legendre stage
  // (leg_tc.cu), p <= 39: [m][K step][digit][Np x 16], offsets per m, row exponents [m][p+1]
  uint16_t* leg_digits = nullptr;
  int* leg_toff = nullptr;
  signed char* leg_exp = nullptr;
};

struct Drop {
  int p = 0, q = 0;
  int64_t coef_off = 0;      // into scalar coefficient vectors
  int64_t tgt_off = 0;       // into target arrays
  int64_t src_off = 0;       // into source arrays
  int nt = 0, ns = 0, nc = 0;
  double lam = 1.0;
  double centre[3] = {0, 0, 0};
  DegreeTables* tab = nullptr;
  // singular rows as two FP32 planes (hi, then lo = value - hi): the FP32 path reads the hi plane
  // only, the FP64-class path both (double-float); same bytes as FP64 storage
  float* rows_lap = nullptr;    // [2][nt][kNumLap][nc]
  float* rows_sto = nullptr;    // [2][nt][kNumSto][nc]
};

// The drops of one degree, wherever they lie in the layout: transforms over a list take one launch per
// distinct degree. Entry l is drop idx[l]; its scalar coefficients start at coef_off[l] (vector fields
// at 3 coef_off[l]) and its grid values at val_off[l] (a source, target or upsampled-grid offset).
struct DropList {
  const int* idx = nullptr;
  const int64_t* coef_off = nullptr;
  const int64_t* val_off = nullptr;
};

// Per-drop description read by the kernels.
struct DropDev {
  int p, q, nt, ns, nc;
  int64_t coef_off, tgt_off, src_off;
  double lam;
  double cx, cy, cz;
  const float* rows_lap;        // [2][nt][kNumLap][nc] (hi plane, lo plane)
  const float* rows_sto;        // [2][nt][kNumSto][nc]
};

// Target tile of the all-pairs kernels: targets [t0, t0+nt) of one drop.
struct PairTile {
  int drop;
  int t0;      // global target index
  int nt;
};

// Drops grouped by degree (set up with the layout): device lists with source and target offsets.
struct DegreeGroup {
  DegreeTables* tab = nullptr;
  int n = 0;                 // drops of this degree
  int first = 0;             // first of them in the layout (for host-side per-drop data)
  int* idx = nullptr;        // [n] device
  int64_t* coef = nullptr;   // [n] device
  int64_t* src = nullptr;    // [n] device
  int64_t* tgt = nullptr;    // [n] device
  int64_t* tgt3 = nullptr;   // [n] device: 3 tgt (vector fields on the targets, component-major per drop)
  DropList sources() const { return DropList{idx, coef, src}; }
  DropList targets() const { return DropList{idx, coef, tgt}; }
  DropList targets3() const { return DropList{idx, coef, tgt3}; }
};

struct Geometry {
  // targets (FP64, SoA): x y z nx ny nz J, each [ntarget]
  double* tgt = nullptr;
  // sources (FP64, SoA): x y z nx ny nz w(=omega J), each [nsource]
  double* src = nullptr;
  // FP32 copies relative to the drop centre: targets (hi) and sources
  float* tgt32 = nullptr;   // x y z nx ny nz  relative position + normal, each [ntarget]
  float* src32 = nullptr;   // x y z nx ny nz w, each [nsource]
  float* src32lo = nullptr; // low parts: value - (double)src32, same layout (double-float sums)
  // positions relative to the drop centre split on the quantum 2^-Q of the FP64-class pair sums
  // (pair_dq.cuh): [xq yq zq][xl yl zl], each [nsource]
  float* srcq = nullptr;
  int* tgt_drop = nullptr;  // [ntarget]
  double* centres = nullptr;// [n_drops][3]
  int64_t* src_start = nullptr;  // [n_drops+1]
};

}  // namespace shbim

struct shbim_ctx {
  shbim_opts opts{};
  std::string err;
  int n_drops = 0;
  int64_t ncoef = 0, ntarget = 0, nsource = 0;
  std::vector<shbim::Drop> drops;
  std::map<int, shbim::DegreeTables*> tables;
  shbim::Geometry geo;
  std::vector<shbim::PairTile> tiles;
  std::vector<shbim::DegreeGroup> groups;  // drops by degree, in order of first appearance
  shbim::PairTile* tiles_dev = nullptr;
  double* lamm1_dev = nullptr;    // lambda_j - 1 per drop
  shbim::DropDev* drops_dev = nullptr;
  int pair_splits = 1;            // default source-split count of the layout
  int split_max = 1;              // capacity of the partial-sum buffer in splits
  // shape of the FP32 all-pairs launches per kernel kind (Laplace DL, Laplace SL, Stokes S + D, Stokes S,
  // Stokes D):
  // targets per thread and source splits, autotuned on the first launch of a layout
  struct PairCfg {
    int tpt = 1;
    int splits = 1;
    bool tuned = false;
    bool queue = false;           // persistent CTAs on an atomic work counter
    int fp64class_splits = 0;     // source splits of the FP64-class kernel (0: not chosen yet)
  } pair_cfg[5];
  int* pair_queue = nullptr;      // [2] work counter and finished-CTA count (zero between launches)
  bool autotune = true;           // off: every layout keeps the default launch shape
  // the double-float row build's two lanes (chunks alternate between the caller's stream and the
  // side stream): per lane the rotated positions, weights, Fourier output, rows, position copy
  // (of drop xdrop) and row exponents, sized in doubles
  struct RowLane {
    double *rot = nullptr, *w = nullptr, *F = nullptr, *v = nullptr, *xdf = nullptr, *rexp = nullptr;
    size_t rot_n = 0, w_n = 0, F_n = 0, v_n = 0, xdf_n = 0, rexp_n = 0;
    int xdrop = -1;
  } lanes[2];
  float* dens_split = nullptr;    // [2][3 ncoef] hi / lo planes of a density for the self GEMV
  size_t dens_split_cap = 0;
  int outer_prec = SHBIM_PREC_DF64;  // FP64-class applications: refinement residuals, one-shot sums
  int rows_prec = SHBIM_PREC_DF64;   // arithmetic of the singular-row build (FP64 or double-float)
  int self_prec = SHBIM_PREC_DF64;   // self-row application in FP32 mode: both planes (double-float) or hi only
  int oneshot_prec = SHBIM_PREC_DF64;  // one-shot applications of shbim_rates in FP32 mode
  // shape G of the linear part of the far field E_u + E_q G x (symmetric, traceless):
  // xx, xy, xz, yy, yz, zz
  double field_g[6] = {1.0, 0.0, 0.0, -1.0, 0.0, 0.0};
  // Stokes preconditioner (gmres.cu): per drop an orthonormal basis of its six rigid-body motions and
  // its normal mode, [7][3 nc] at 7 * 3 coef_off (FP64, rebuilt per geometry), and the drop's factors
  bool stokes_prec = true;
  double* prec_basis = nullptr;
  double* prec_dots = nullptr;    // [n_drops][7]
  double* prec_fac = nullptr;     // [n_drops][6]: inverse (1/(lam+1), 1/2 - ., 1/(2 lam) - .), forward (lam+1, ...)
  bool dq_pairs = true;           // FP64-class pair sums on quantised positions (k_pairs_dq) or general double-float
  double dq_scale = 0.0;          // 2^Q of the quantised positions (0: not built for this geometry)
  unsigned* dq_ext_dev = nullptr; // [n_drops] largest |x - c| over each drop's sources (float bits)
  unsigned char* dq_far = nullptr; // [n_drops][n_drops]: the drop pair uses the quantised form
  int dq_cap = 0;                 // drops the two tables above hold
  int eos = SHBIM_EOS_LANGMUIR;      // tension law of shbim_rates / shbim_step (shbim_set_equation_of_state)
  bool refine_direct[2] = {true, true};     // refined solves (electric, Stokes): first inner solve aims at the end
  shbim_mlp* warm_net = nullptr;  // learned initial guesses of shbim_rates (shbim_set_warm_start), not owned
  const double* xcoef_cur = nullptr;  // position coefficients of the current geometry (during a rates call)
  bool tc_rows = true;            // double-float build: Fourier analysis on the tensor cores
  bool tc_rot = true;             // ... and the degree-block rotations (rot_tc.cu)
  bool tc_leg = true;             // ... and the Legendre stage of the analysis (leg_tc.cu)
  int* tc_err = nullptr;          // device flag: a tensor-core kernel timed out
  uint64_t wait_ns = 1000000000ull;  // limit of every bounded wait inside a kernel (nanoseconds)
  // workspaces
  double* dens_up = nullptr;      // [3][nsource] source strengths (FP64)
  float* dens_up32 = nullptr;     // [6][nsource] source strengths (FP32)
  float* dens_up32lo = nullptr;   // [6][nsource] low parts of the strengths (double-float sums)
  double* part = nullptr;         // [pair_splits][3][ntarget] partial sums
  double* grid_out = nullptr;     // [3][ntarget] operator values before projection
  double* xup = nullptr;          // per drop [3][kNumTab][ns]: position and derivatives on the up grid
  double* sht_scratch = nullptr;  // Fourier stage of forward transforms
  size_t sht_scratch_elems = 0;
  // singular-row build workspace
  double* rot_coef = nullptr;
  double* wbuf = nullptr;
  double* vbuf = nullptr;
  size_t rot_elems = 0, wbuf_elems = 0, vbuf_elems = 0;
  // GMRES
  struct Gmres {
    int sys = -1;
    int64_t n = 0;
    int m = 50;
    double* V = nullptr;        // [m+1][n]
    double* w = nullptr;        // [n]
    double* x = nullptr;        // [n]
    double* b = nullptr;        // [n]
    double* h = nullptr;        // [2][m+2] device dots
    double* h_host = nullptr;   // pinned
    double* Av = nullptr;       // [n] operator output
    double* diag = nullptr;     // [n] identity part of the system (diffusion: M^{-1})
    double* y = nullptr;        // [m] least-squares solution uploaded for x updates
    double offdiag = 0.0;       // factor of the layer operator in the system
    double* xr = nullptr;       // [n] refinement: outer iterate
    double* rr = nullptr;       // [n] refinement: outer residual
    double* dr = nullptr;       // [n] refinement: correction
    double* tmp = nullptr;      // [n] preconditioned vector (diffusion: M^{-1} v; Stokes: P^{-1} v)
    bool prec = false;          // Stokes system solved right-preconditioned (iterate y = P x)
    bool raw = false;           // the next applications are of the system itself (refinement residuals)
    double* dstate = nullptr;   // device cycle state: H [(m+1) m], cs [m], sn [m], g [m+1], y [m], scalars [8]
    int* istate = nullptr;      // device cycle state: k, total, flags, spare
    double* vstage = nullptr;   // [n] operator input staged for the device cycle
    std::vector<double> H;      // (m+1) x m, column-major k*(m+1)+i
    std::vector<double> cs, sn, g;
    int k = 0;                  // Arnoldi steps in the current cycle
    int total = 0;
    double bnorm = 0.0;
    double resid = 1.0;
    int64_t cap = 0;
  } gm;
  // nearly-singular correction (near.cu)
  struct Near {
    bool enabled = true;
    int npairs = 0;
    double min_dist = INFINITY;   // smallest near-target distance to another drop's upsampled nodes
    double min_ratio = INFINITY;  // the same in units of that drop's spacing h_j
    double* stats = nullptr;  size_t stats_cap = 0;
    int64_t* det_t = nullptr; size_t det_t_cap = 0;
    int* det_j = nullptr;     size_t det_j_cap = 0;
    int64_t* pair_t = nullptr; size_t pair_t_cap = 0;
    int* pair_j = nullptr;    size_t pair_j_cap = 0;
    double* fgeo = nullptr;   size_t fgeo_cap = 0;    // [7][nfine] upsampled x, n, w
    float* fgeo32 = nullptr;  size_t fgeo32_cap = 0;  // same, positions relative to the centre
    double* fstr = nullptr;   size_t fstr_cap = 0;    // [6][nfine] upsampled strengths
    float* fstr32 = nullptr;  size_t fstr32_cap = 0;
    float* fgeo32lo = nullptr;  size_t fgeo32lo_cap = 0;  // low parts (double-float sums)
    float* fstr32lo = nullptr;  size_t fstr32lo_cap = 0;
    int64_t* foff_dev = nullptr; size_t foff_cap = 0; // [2][n_drops]: offset, count
    int4* groups = nullptr;   size_t groups_cap = 0;  // runs of <= 128 pairs sharing a source drop:
    int ngroups = 0;                                  // (first pair, count, drop, 0)
    std::vector<int64_t> fine_off_h, fine_n_h;
    int64_t nfine = 0;
    // drops with near targets grouped by degree (one upsampled-strength launch per degree): device
    // lists of drop index, coefficient offset and upsampled-grid offset
    struct DegGroup {
      shbim::DegreeTables* tab = nullptr;
      int n = 0;
      int* idx = nullptr;
      int64_t* coef = nullptr;
      int64_t* fine = nullptr;
    };
    std::vector<DegGroup> groups_d;
  } near;
  // physics workspaces (forces, rates, step state)
  struct Phys {
    double* buf = nullptr;
    size_t cap = 0;
    double* grid = nullptr;
    size_t grid_cap = 0;
    double* state = nullptr;
    size_t state_cap = 0;
    double* lb = nullptr;       // surface Laplacian workspace [6][nsource]
    size_t lb_cap = 0;
    float* feat = nullptr;      // learned warm start: features [feature count]
    size_t feat_cap = 0;
    double* guess = nullptr;    // learned warm start: E_n and u guesses [4 ncoef]
    size_t guess_cap = 0;
    double* rep = nullptr;      // reparametrisation workspace
    size_t rep_cap = 0;
  } phys;
  int64_t launches = 0;
  int64_t applications = 0;
  // CUDA graphs of the GMRES operator application, per (system, precision), re-captured per
  // geometry on a library-owned stream and replayed on the caller's stream
  bool graphs_on = true;
  int64_t geom_version = 0;
  cudaStream_t cap_stream = nullptr;
  // second library stream for the concurrent branches of an operator application (self rows
  // and near-field correction beside the all-pairs sums), with its fork/join events
  bool concurrent = true;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_coarse = nullptr, ev_join = nullptr;
  struct MatvecGraph {
    cudaGraphExec_t exec = nullptr;
    double* in = nullptr;
    double* out = nullptr;
    int64_t n = 0;
    int64_t version = -1;
    int64_t kernels = 0;   // kernel nodes per replay
    bool warm = false;
  } graphs[9];                    // [system][precision]
  // GMRES cycles run on the device: one graph per (system, precision, geometry) whose conditional
  // 'while' node repeats an Arnoldi step -- operator application, two classical Gram-Schmidt passes,
  // normalisation, Givens rotation and the convergence test, all in kernels -- until the residual
  // estimate reaches the tolerance, the Krylov space is full or the step budget is spent; then the
  // least-squares solution and the update of x. The host reads the state back once per cycle.
  struct CycleGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t version = -1;
    int64_t n = 0;
    int m = 0;
    int64_t body_kernels = 0;     // kernel launches per Arnoldi step
    bool failed = false;          // building failed once: host-driven steps for this slot
  } cycles[9];
  bool device_gmres = true;       // shbim_gmres_solve runs its cycles as device graphs
  double diff_c = 0.0;            // coefficient of the diffusion system
  // optional per-class kernel timing
  bool timing = false;
  struct TimedRange {
    int cls;
    cudaEvent_t a, b;
    double work;                // algorithmic flops of the bracketed launch (pair classes)
  };
  std::vector<TimedRange> timed;
  std::vector<cudaEvent_t> event_pool;
  double class_ms[SHBIM_K_COUNT] = {0};
  int64_t class_launches[SHBIM_K_COUNT] = {0};
  double class_work[SHBIM_K_COUNT] = {0};
  int64_t cross_pairs = 0;        // target-source pairs of different drops per all-pairs launch
};

namespace shbim {

// ---- error helpers
int fail(shbim_ctx* ctx, int code, const std::string& msg);
int cuda_fail(shbim_ctx* ctx, cudaError_t e, const char* what);
#define SHBIM_CHECK_LAUNCH(ctx, what)                                 \
  do {                                                                \
    (ctx)->launches++;                                                \
    cudaError_t e_ = cudaGetLastError();                              \
    if (e_ != cudaSuccess) return ::shbim::cuda_fail((ctx), e_, what);\
  } while (0)
#define SHBIM_CUDA(ctx, call)                                         \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return ::shbim::cuda_fail((ctx), e_, #call);\
  } while (0)

// ---- timing: bracket a launch of class `cls` on stream s (no-op unless timing is on)
struct TimeScope {
  shbim_ctx* ctx;
  int cls;
  cudaStream_t s;
  cudaEvent_t b = nullptr;
  double work = 0.0;            // algorithmic flops of what the scope brackets (set by the caller)
  TimeScope(shbim_ctx* c, int k, cudaStream_t st);
  ~TimeScope();
};

// ---- tables (tables.cu)
int build_degree_tables(shbim_ctx* ctx, int p, DegreeTables** out);
void free_degree_tables(DegreeTables* t);

// ---- transforms (sht.cu)
// Synthesis: for n_items coefficient vectors of degree p, values on grid g for the
// requested kinds (bit 0 value, bit 1 d/dtheta, bit 2 (1/sin) d/dphi).
// out[item * item_stride + kind_slot * kind_stride + node]; kinds are packed in order.
// If scale != nullptr, each node value is multiplied by scale[node] (values only).
// If out32 != nullptr the result is also written as float to out32 at the same index.
// With a drop list L: n_items = L's length x kpd, item l kpd + c reads coef + kpd L.coef_off[l] +
// c coef_stride and writes out + L.val_off[l] + c item_stride (+ kind slot * kind_stride).
int sht_synth(shbim_ctx* ctx, const GridTables& g, int n_items, const double* coef,
              int64_t coef_stride, int kinds, double* out, int64_t item_stride,
              int64_t kind_stride, const double* scale, float* out32, cudaStream_t s,
              int kpd = 0, const DropList* L = nullptr);
// out32lo (optional) receives value - (double)out32 as float (the low part of a double-float copy)
int sht_synth_scaled(shbim_ctx* ctx, const GridTables& g, int n_items, const double* coef,
                     int64_t coef_stride, double* out, int64_t item_stride, const double* scale,
                     double alpha, float* out32, cudaStream_t s, float* out32lo = nullptr);
// With a drop list L (non-null), the nb drops are L's entries instead of consecutive drops: coef, out,
// scale and alpha_drop are then the bases of the whole layout's arrays (drop_stride is unused).
int sht_synth_drops(shbim_ctx* ctx, const GridTables& g, int nb, int kpd, const double* coef, int64_t coef_stride,
                    double* out, int64_t comp_stride, int64_t drop_stride, const double* scale, double alpha,
                    const double* alpha_drop, float* out32, cudaStream_t s, float* out32lo = nullptr,
                    const DropList* L = nullptr);
// Analysis: coef[item] = sum_nodes w(node) vals[item][node] S_nm(node) with w = omega_j when
// weighted, else 1. Uses ctx->sht_scratch (grown as needed).
// With a drop list L, n_items = L's length x kpd: item l kpd + c reads vals + L.val_off[l] + c val_stride
// and writes coef + kpd L.coef_off[l] + c coef_stride.
int sht_analysis(shbim_ctx* ctx, const GridTables& g, int n_items, const double* vals,
                 int64_t val_stride, bool weighted, double* coef, int64_t coef_stride,
                 cudaStream_t s, int kpd = 1, const DropList* L = nullptr);

// ---- geometry / singular rows (singular.cu)
int build_geometry(shbim_ctx* ctx, const double* xcoef_dev, cudaStream_t s);
int build_singular_rows(shbim_ctx* ctx, const double* xcoef_dev, cudaStream_t s);
// the same rows computed in double-float arithmetic on the FP32 pipe (singular_df.cu)
int build_singular_rows_df(shbim_ctx* ctx, cudaStream_t s, const double* xcoef_dev);
int ensure_side_stream(shbim_ctx* ctx);
// out[t] (+)= self rows . density for every target (scalar Laplace kind or Stokes tensors).
int apply_self_laplace(shbim_ctx* ctx, int which, const double* dens, double* out, cudaStream_t s);
int apply_self_stokes(shbim_ctx* ctx, const double* f, const double* u, double* out,
                      cudaStream_t s);

// ---- nearly-singular correction (near.cu)
int build_near(shbim_ctx* ctx, const double* xcoef, cudaStream_t s);
int apply_near_laplace(shbim_ctx* ctx, int which, const double* dens, double* out, cudaStream_t s,
                       cudaEvent_t before_sums = nullptr);
int apply_near_stokes(shbim_ctx* ctx, const double* f, const double* u, double* out, cudaStream_t s,
                      cudaEvent_t before_sums = nullptr);
// geometry (x, n, w = omega J) of a grid from its synthesised x, x_theta, x_phi/sin (singular.cu)
int geometry_kernel(shbim_ctx* ctx, const double* buf, int64_t n, int nkind, const GridTables& g, double* out,
                    int64_t ld, int64_t off, cudaStream_t s);
int geometry_kernel32(shbim_ctx* ctx, const double* buf, int64_t n, int nkind, const GridTables& g, double* out,
                      float* out32, int64_t ld, int64_t off, const double* centre, cudaStream_t s,
                      float* out32lo = nullptr);

// ---- surface Laplacian (physics.cu)
int laplace_beltrami(shbim_ctx* ctx, const double* coef, double* out, cudaStream_t s);

// ---- tensor-core Fourier analysis of double-float rows (dft_tc.cu)
// F[r][cs][m] = sum_k W[r][k] (cos|sin)(m phi_k), r < rows, on drop d's degree 2p+1 grid; W and F
// double-float (float2), W rows of 2q+2 values, F rows of 2(p+1) values.
// highest degree the tensor-core rotations take for drops of degree p (-1: none)
int rot_tc_nmax(int p);
int rot_tc_digits(shbim_ctx* ctx, int p, const std::vector<double>& D, const std::vector<double>& theta,
                  DegreeTables& T);
int rotate_tc(shbim_ctx* ctx, const DegreeTables& T, bool adjoint, const float2* vin, int64_t in_stride, int nc,
              int t_begin, int ct, int ncomp, float2* vout, float* rows_lap, float* rows_sto, int nt_drop,
              cudaStream_t s);
int dft_tc_digits(shbim_ctx* ctx, int p, DegreeTables& T);
// the kernel holds a 128-row tile of W in shared memory: degrees up to 34
bool dft_tc_fits(int p);
int analysis_fourier_tc(shbim_ctx* ctx, const DegreeTables& T, const float2* W, int64_t rows, const int* rexp,
                        float2* F, cudaStream_t s, bool omajor = false);
bool leg_tc_fits(int p);
int leg_tc_digits(shbim_ctx* ctx, int p, const std::vector<double>& alf0, DegreeTables& T);
int analysis_legendre_tc(shbim_ctx* ctx, const DegreeTables& T, const float2* FT, int64_t nitems, float2* coef,
                         int64_t coef_stride, cudaStream_t s);

// ---- shape-dependent state for an unchanged layout (api.cu)
int rebuild_geometry(shbim_ctx* ctx, const double* xcoef_dev, cudaStream_t s);

// ---- all-pairs sums (pairs.cu)
// the sums go to partial buffers; `before_reduce` (optional) is waited for before they are
// added into out_accum
// Stokes preconditioner basis and factors of the current geometry (gmres.cu)
int build_stokes_preconditioner(shbim_ctx* ctx, const double* xcoef_dev, cudaStream_t s);
// quantised source positions of the FP64-class pair sums (once per geometry)
int build_quantized_sources(shbim_ctx* ctx, cudaStream_t s);
int pairs_laplace(shbim_ctx* ctx, int which, double* out_accum, cudaStream_t s, cudaEvent_t before_reduce = nullptr);
int pairs_stokes(shbim_ctx* ctx, bool has_f, bool has_u, double* out_accum, cudaStream_t s,
                 cudaEvent_t before_reduce = nullptr);
// algorithmic flops of one all-pairs launch: cross pairs times the operations of one kernel term
// (kind 0 Laplace DL, 1 SL, 2 Stokes S + D, 3 S, 4 D)
double pairs_work(const shbim_ctx* ctx, int kind);


}  // namespace shbim
