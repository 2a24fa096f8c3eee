// Host-side objects and the launchers that one translation unit exposes to another.
#pragma once

#include "common.cuh"

namespace gnp {

// Weight views inside the flat blob (float32, layout in include/gnp.h).
constexpr int D = GNP_D;
constexpr int HID = GNP_MLP_HIDDEN;
constexpr int ENC_W1 = 0, ENC_B1 = 32, ENC_W2 = 64, ENC_B2 = 64 + 512;
constexpr int ENC_COUNT = 592;
constexpr int LAYER_COUNT = 512;
constexpr int DEC_COUNT = 577;
inline int layer_off(int l) { return ENC_COUNT + l * LAYER_COUNT; }
inline int dec_off(int L) { return ENC_COUNT + L * LAYER_COUNT; }
inline int weight_count(int L) { return ENC_COUNT + L * LAYER_COUNT + DEC_COUNT; }

// Kernel-parameter copies of the weights: passed by value (__grid_constant__), so the
// epilogues read them as uniform constant-bank operands.
struct __align__(16) EncW { float W1[32]; float b1[32]; float W2[512]; float b2[16]; };
struct __align__(16) LayerW { float U[256]; float W[256]; };
struct __align__(16) DecW { float W1[512]; float b1[32]; float W2[32]; float b2; };
// Transposed copies for the short-row kernels' paired (f32x2) products: WT[k*16 + c] =
// W[c*16 + k] (and UT from U), DT1[k*16 + c] = decoder W1[c*32 + k], so that the weights of
// two consecutive inputs c, c+1 of one output k sit side by side.
struct __align__(16) LayerWT { float WT[256]; float UT[256]; };
struct __align__(16) DecWT { float DT1[512]; float b1[32]; float W2[32]; float b2; };

// Indexed vector inside a basis: base + (*jptr + off) * stride (jptr may be null).
struct ColPtr {
  void* base;
  size_t stride;
  const int* jptr;
  int off;
};

struct TrainState;  // train.cu
struct Server;      // serve.cu
struct DevState;    // solver.h

// The FGMRES step whose basis vector the next GNP application forms itself (Algorithm 1):
// after the CGS2 passes of step j = st->jv, v_{j+1} = (w1 - V_j h2) / h_{j+1,j} with
// h_{j+1,j} = sqrt(||w1||^2 - ||h2||^2), and the step's Givens update still to do.
struct VNext {
  double* V;
  const double* w;
  const double* h1;
  const double* h2;
  DevState* st;
  double* H;
  double* R;
  double* cs;
  double* sn;
  double* g;
  double* hist;
  unsigned long long* thist;
  // Overlapped CGS2 (dcgs = 1): h1 holds a_s = V_{s-1}^T v'_s, h2 the first-pass h_s
  // = V_s^T w_s, hf the finished column s-1; the encoder forms v'_{s+1} = (w_s - V_s h_s)
  // / rho_s and encodes it (no finishing block: the reorthogonalisation branch finishes
  // the columns).
  const double* hf;
  int dcgs;
};

// Mutable scratch of one GNP application: hidden ping-pong blocks (n x 16 float32 each,
// also used as bfloat16), the norm tau and the reduction scratch.  A model owns one;
// a server slot owns another, so that one model may serve several concurrent solves.
struct ApplyWs {
  void* H[2] = {nullptr, nullptr};
  double* tau = nullptr;
  RedScratch red;
};
int apply_ws_alloc(ApplyWs& ws, int n);
void apply_ws_free(ApplyWs& ws);
inline size_t apply_ws_bytes(int n) { return (size_t)n * 16 * 4 * 2 + 16 + (size_t)4 * NUM_SMS_GB300 * 8 + 8; }

// CSC (transpose) of a matrix, built on the device once (train and gamma use it).
int mat_build_csc(gnp_mat* A, cudaStream_t st);

// y = A x (float64 values), x in float64 or float32 (xf).  Tile SpMV kernel.
int spmv_launch(const gnp_mat* A, const double* x, const float* xf, double* y, cudaStream_t st);

}  // namespace gnp

struct gnp_model {
  gnp_mat* A = nullptr;
  gnp_config cfg{};
  int hprec = GNP_H_FP32;
  double gamma = 0.0;
  float* valhat = nullptr;        // [nnz] A/gamma in the CSR order
  float* valhat_t = nullptr;      // [nnz] A/gamma in the CSC order (training)
  std::vector<float> w_host;      // weights used to build kernel parameters
  bool host_stale = false;        // device weights changed by training
  float* w_dev = nullptr;         // [count] training copy
  float* w_best = nullptr;        // [count] best-loss snapshot
  gnp::ApplyWs ws;                // the model's own apply scratch
  gnp::TrainState* train = nullptr;
  unsigned long long version = 1; // bumped whenever weights or hprec change
};

namespace gnp {

// z = M(v) on `st`.  v: column of a basis (may be scaled in place first by 1/(*vscale)
// when vscale is non-null: the FGMRES step normalises v_{j} inside the same pass).
// ctl (may be null): device {j, active}; when active == 0 every kernel returns at once.
// z: float32 output column; trace: optional float32 [(L+1)*n*16].
// ev (may be null): 2*L events; ev[2l] / ev[2l+1] are recorded on `st` just before /
// after the launch of layer l's Res-GCONV kernel (the timing of the hot kernel).
// vn (may be null): the encoder first forms the pending basis vector of that FGMRES step
// (written to V[:, jv+1], normalised) and encodes it, while one extra block finishes the
// step (v and vscale are then unused).
// fork (may be null): recorded on `st` right after the encoder, and `side` made to wait
// for it, so that work launched on `side` next overlaps the Res-GCONV layers.
int apply_launch(gnp_model* M, ColPtr v, const double* vscale, ColPtr z, float* trace,
                 const int* ctl, cudaStream_t st, cudaEvent_t* ev = nullptr,
                 const ApplyWs* ws = nullptr, const VNext* vn = nullptr, cudaEvent_t fork = nullptr,
                 cudaStream_t side = nullptr);

// Kernel-parameter copies of the encoder/decoder and of layer l's weights.
void fill_enc_dec(const std::vector<float>& w, int L, EncW& ew, DecW& dw);
void fill_layer_w(const std::vector<float>& w, int l, LayerW& lw);
void fill_layer_wt(const std::vector<float>& w, int l, LayerWT& lw);
void fill_dec_wt(const std::vector<float>& w, int L, DecWT& dw);

// The L Res-GCONV layers of a K-system GNP on the short-row kernels (multi-right-hand-side
// FGMRES), when multi_row_ok(M): hidden blocks [n K, 16] float32, z = column zp ([n][K]).
bool multi_row_ok(const gnp_model* M);
int multi_row_layers(gnp_model* M, int K, float* H0, float* H1, ColPtr zp, const double* tau_one, const int* ctl,
                     cudaStream_t st);

// The TMA-gather Res-GCONV layer (gconv_tma.cu), for matrices with rows too long for the
// short-row kernels.  tma_prepare builds the matrix's schedules (host, synchronous; call
// before any stream capture); tma_active says whether the layers use it (schedule built
// and GNP_GCONV_TMA=1 in the environment).  tma_layer_launch: one layer Hin -> Hout, or
// with dec the decoder-fused last layer Hin -> z (column zp, tau for tau / sqrt(n)).
int tma_prepare(gnp_mat* A);
bool tma_active(const gnp_mat* A);
void tma_sched_free(TmaSched& s);
template <class HT>
int tma_layer_launch(const gnp_mat* A, int form, bool dec, const float* valhat, const HT* Hin, HT* Hout, ColPtr zp,
                     const double* tau, double sqrt_n, const int* ctl, const LayerW& lw, const DecW& dw,
                     cudaStream_t st);

// ---------------------------------------------------------------- grouped steps (serving)
//
// One request of the grouped solve server, as its kernels see it (a device array indexed by
// slot): its matrix, its GNP scratch and its FGMRES workspace.  A grouped launch runs the
// same kernel body for several requests at once: its blocks are the requests' own grids
// laid end to end (GTable), each block working on its request's data with the block index
// and count that request's stand-alone launch would have, so every request computes
// exactly what a lone solve computes.
// A grouped request's place in its cycle and its stopping rules, kept on the device (not in
// DevState, which the step kernels load and store whole): phase = the round's index in
// the cycle (0..m, set by the round's encoder; -1 before the first round), the counters of
// cycle_after, and done / status once the rules end the solve.
struct GCtl {
  int phase, done, status, stagn, mism, restarts, cycles, pad;
};

struct GSlot {
  GCtl* gc;
  int m;
  const int* rp;
  const int* col;
  const double* val;
  const float* valhat;  // A_hat = A / gamma (float32)
  int n, L, noscale;
  double sqrt_n;
  void* Hh[2];  // hidden ping-pong blocks
  double* tau;
  double* V;
  float* Z;
  double* w;
  DevState* st;
  double* Hb;  // H_bar
  double* R;
  double* cs;
  double* sn;
  double* g;
  double* h1;
  double* h2;
  double* hf;
  double* hist;
  unsigned long long* thist;
  double* partials;
  unsigned* counter;
  const double* b;
  double* x;
};

// Requests per grouped GNP launch: each request's weights ride in the launch's kernel
// parameters (the decoder-fused layer carries a layer's and the decoder's, 4.4 KB), so that
// the epilogues read them as constant-bank operands as the stand-alone kernels do.
constexpr int GW = 6;

// Host view of one grouped request: its slot in the device array, size and model.
struct GHost {
  int slot;
  int n;
  const gnp_model* M;
};

// Whether a request with preconditioner M can run in grouped steps (the short-row layer
// kernels with four lanes per row, L >= 1).
bool grouped_ok(const gnp_model* M);
// z = M(v) of the current FGMRES step for every request of `reqs` (one hidden precision
// and layer form): the encoder (forming v_j and finishing step j-1, or v_0 = r / beta at a
// cycle's first step), the L-1 Res-GCONV layers and the decoder-fused last layer.
int grouped_apply_launch(const std::vector<GHost>& reqs, const GSlot* d_slots, cudaStream_t st);
// The rest of the step for every request: w = A z with CGS2 pass 1, then pass 2.
int grouped_krylov_launch(const std::vector<GHost>& reqs, const GSlot* d_slots, cudaStream_t st);
// Cycle end for the requests of `reqs` that reach it this round (phase m): x += Z y,
// r = b - A x, beta, the stopping rules, and the restart or the end of the solve.
int grouped_cycle_end_launch(const std::vector<GHost>& reqs, int m, const GSlot* d_slots, cudaStream_t st);
// Work tables: entries (slot, blocks) in order, at most `cap` per table.
std::vector<GTable> gt_build(const std::vector<std::pair<int, int>>& entries, int cap);

// Make the host copy of the weights current (after training).
int model_sync_host(gnp_model* M);
// Everything apply_launch needs that is not a stream operation (host weights, kernel
// attributes); call before capturing apply_launch into a CUDA graph.
int apply_prepare(gnp_model* M);
unsigned long long model_version(const gnp_model* M);
int gamma_launch(gnp_mat* A, double* gamma_dev, cudaStream_t st);
void solver_free(Solver* s);
void multi_solver_free(MultiSolver* s);
int solver_create(int n, int m, int maxiters, Solver** out);
size_t solver_bytes(int n, int m, int maxiters);
void train_reset(TrainState* t);
void train_free(TrainState* t);

}  // namespace gnp
