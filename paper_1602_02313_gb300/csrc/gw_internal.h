// Internal declarations of libgw (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gw.h"

#ifdef __CUDACC__
#include <cuda_runtime.h>
#else
typedef struct CUstream_st* cudaStream_t;
typedef struct CUevent_st* cudaEvent_t;
#endif

namespace gwi {

struct Transforms {
  std::vector<double> B_fwd;       // cplx [nnu][ntau]
  std::vector<double> F_fwd;       // cplx [nw][ntau]
  std::vector<double> F_cont;      // cplx [ncont][ntau]
  std::vector<double> B_bwd;       // real [ntau][2 nnu]
  std::vector<double> F_bwd;       // real [ntau][2 nw]
  std::vector<double> F_bwd_beta;  // real [2 nw]: value at tau = beta^-
};

void build_transforms(const std::vector<double>& tau, const std::vector<double>& poles, double beta,
                      const std::vector<int>& nu_idx, const std::vector<int>& w_idx, int ncont,
                      Transforms* out);

// Split-precision operand copies for the tensor-core contractions of one q.
struct MixedWork {
  int iq = -1;                // q whose M slices are staged (-1: none)
  int prec = -1;
  void* mslices = nullptr;    // per-precision staged copy of M[q]
  size_t mslices_bytes = 0;
  void* wslices = nullptr;    // per-tau split copies of W~ (Sigma) or scaled rows (P)
  size_t wslices_bytes = 0;
  double* dacc = nullptr;     // P strip metadata (uploaded once per context) and error word
  size_t dacc_bytes = 0;
  bool strips_ready = false;
  int strips_form = -1;       // the form the uploaded strips were built for
};

}  // namespace gwi

struct gw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // grid
  double beta = 0;
  int ntau = 0, npole = 0, nnu = 0, nw = 0, ncont = 0;
  std::vector<double> tau, poles;
  std::vector<int> nu_idx, w_idx;
  gwi::Transforms T;
  // system
  uint64_t seed = 0;
  int q0 = 0;
  int64_t launches = 0;
  int nk = 0, nq = 0, nb = 0, nocc = 0, ni = 0;
  double omega = 1.0;
  std::vector<int> kmq;
  std::vector<double> v;
  // device copies
  int* d_kmq = nullptr;        // [nq][nk]
  int* d_widx = nullptr;       // [nw]
  double* d_tau = nullptr;     // [ntau]
  double* d_sqrtv = nullptr;   // [nq][ni]
  double* d_v = nullptr;       // [nq][ni]
  const double* d_M = nullptr; // cplx [nq][nk][ni][nb][nb], or one q's block when m_per_q
  double* d_M_own = nullptr;
  bool m_per_q = false;        // M generated one q at a time into d_M_own
  int m_cur = -1;              // the q whose block d_M_own holds (m_per_q)
  bool m_lazy = false;         // all q kept, each generated on a side stream ahead of first use
  cudaStream_t m_stream = nullptr;
  std::vector<cudaEvent_t> m_done;  // [nq]: generation of M[q] finished (m_lazy)
  std::vector<char> m_issued;       // [nq]
  double* d_Bfwd = nullptr;    // cplx [nnu][ntau]
  double* d_Ffwd = nullptr;    // cplx [nw][ntau]
  double* d_Fcont = nullptr;   // cplx [ncont][ntau]
  double* d_Bbwd = nullptr;    // [ntau][2 nnu]
  double* d_Fbwd = nullptr;    // [ntau][2 nw]
  double* d_Fbwd_beta = nullptr;
  // exchange workspace: vm[k][p] = sum_I v_I |M^I_p|^2
  double* d_vm = nullptr;
  size_t vm_bytes = 0;
  // screening workspace: augmented systems [nsys][ni][2 ni] cplx
  double* d_aug = nullptr;
  size_t aug_bytes = 0;
  // continuation
  int cpe_ngrid = 0;
  std::vector<double> cpe_x;
  double cpe_ridge = 0;
  double* d_cpe_x = nullptr;
  double* d_cpe_A = nullptr;    // real [2 ncont][ngrid]
  double* d_cpe_N = nullptr;    // real [ngrid][ngrid]: A^T A + lambda^2 I
  double* d_cpe_tab = nullptr;
  void* ff_ws = nullptr;        // float-float copies of a bosonic transform's input
  void* d_tsys = nullptr;       // gw_screen_tau: two copies of the augmented system + increments
  size_t tsys_bytes = 0;
  void* d_dm = nullptr;         // gw_dyson_matrix: Sigma^c(i w), eigenpairs, augmented systems, remainders
  size_t dm_bytes = 0;
  void* d_dyt = nullptr;        // gw_dyson_tau: augmented systems of a chunk of states + the mesh
  size_t dyt_bytes = 0;
  size_t ff_ws_bytes = 0;  // real [1201][ngrid]: Re Phi_m on the QP scan grid
  double* d_cpe_b = nullptr;    // [nprob][ngrid]
  size_t cpe_b_bytes = 0;
  int64_t cpe_nprob = 0;       // problems of the last GW_CPE call
  int* d_cpe_iters = nullptr;   // [nprob] Lawson-Hanson outer iterations of the last call
  size_t cpe_iters_bytes = 0;
  double* d_cpe_seed = nullptr; // [nprob][ngrid] warm start for the next GW_CPE call
  size_t cpe_seed_bytes = 0;
  int64_t cpe_seed_nprob = 0;
  double* d_pade = nullptr;     // cplx [nprob][npade] coefficients
  size_t pade_bytes = 0;
  // tensor-core path
  gwi::MixedWork mw;
  int* d_err = nullptr;                     // error word of the bounded device waits (read by gw_sync)
  long long wait_cycles = 4000000000ll;     // clock cycles a tensor-core pipeline wait may take (~2 s)
  int fault_stall = 0;                      // test fault injection: MMA issuers wait on a barrier nothing sets
  int pol_form = 0;                         // polarization cover: 0 by ni, 1 E = Re P + Im P, 2 Re P and Im P
  int pol_seg_chunks = 32;                  // K chunks per FP32 accumulation segment of P (<= 32)
  size_t pol_part_bytes = 8ull << 30;       // FP32 partial strips of P held at once
  // per-kernel timing (gw_kernel_timing): CUDA events recorded around selected launches
  struct KernelEvents {
    const char* name;
    cudaEvent_t begin, end;
  };
  bool ktiming = false;
  std::vector<KernelEvents> kev;
  std::string err;
};

namespace gwi {
// kernels and host launchers (defined in the .cu files)
gw_status check_launch(gw_ctx* c, const char* what);
// bracket a launch with CUDA events on the context's stream while timing is enabled
void kt_begin(gw_ctx* c, const char* name);
void kt_end(gw_ctx* c);
gw_status set_err(gw_ctx* c, gw_status s, const std::string& msg);

gw_status launch_gen_m(gw_ctx* c, double* M);
// device address of M[iq] ([nk][ni][nb][nb] cplx); with per-q generation, (re)generates the
// block first when it holds another q. NULL on a launch error (set in the context).
const double* m_block(gw_ctx* c, int iq);
gw_status launch_green0(gw_ctx* c, const double* eps, double* G, double* occ);
gw_status launch_dyson(gw_ctx* c, const double* eps, const double* sigx, const double* vxc,
                       const double* sigc_iw, double* G, double* occ);
gw_status launch_pol_fp64(gw_ctx* c, int iq, const double* G, double* P);
gw_status launch_pol_mixed(gw_ctx* c, int iq, const double* G, int prec, double* P);
gw_status launch_pol_many(int njobs, gw_ctx* const* ctxs, const int* iqs, const double* const* G, double* const* P);
gw_status launch_transform(gw_ctx* c, int stat, int dir, int prec, int count, int64_t batch, const double* in,
                           double* out);
gw_status launch_screen(gw_ctx* c, int iq0, int nqb, int prec, const double* P, double* W, int* info,
                        double* aug);
gw_status launch_sigma_fp64(gw_ctx* c, int iq, const double* G, const double* W, double* S);
gw_status launch_sigma_mixed(gw_ctx* c, int iq, const double* G, const double* W, int prec, double* S);
gw_status launch_sigx(gw_ctx* c, int iq, const double* occ, double* Sx, bool ff);
gw_status launch_continue(gw_ctx* c, int method, int64_t nprob, const double* sig_iw, const double* eps,
                          const double* sigx, const double* vxc, int nreal, const double* omega_real,
                          double* sig_real, double* e_qp, int* info);
void free_mixed(gw_ctx* c);
}  // namespace gwi
