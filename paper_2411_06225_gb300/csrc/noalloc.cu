// noalloc.cu -- a RandNet prediction entry point that allocates nothing.
//
// rnp_randnet_predict needs a context, and creating a context allocates
// device memory.  Some callers cannot allocate at the time they need a
// prediction: code running where a device allocation would synchronise the
// device or is forbidden (a real-time loop with a pre-planned memory budget,
// a host callback enqueued on a stream, an embedding application that hands
// out only fixed buffers).  rnp_randnet_predict_noalloc serves them: the
// caller passes the dataset, the weights, the query and the output buffer,
// and the intermediate values (scaled query, features, distance partials,
// ridge coefficients) live in one file-scope device array below, of fixed
// size, that every GPU loading this library keeps until the process exits.
#include "rnp_internal.h"

namespace rnp {

// Limits of the scratch array.
static const long long kNaMaxD = 262144;  // unknowns per state
static const int kNaMaxP = 4096;          // stored pairs
static const int kNaMaxM = 1024;          // hidden neurons

// Layout (doubles): scaled query [maxD] | feature partials [maxM * maxFeatCh]
// | phi_q [maxM] | distance partials [maxP * maxNnCh] | distances [maxP]
// | alpha [RNP_MAX_M] | scale c [3] | scale r [3]; then ints: P, meff,
// idx [RNP_MAX_M], flags [4].
static const long long kNaFeatCh = (kNaMaxD + 1023) / 1024;
static const long long kNaNnCh = 32;  // nn_chunks(d) <= 32 for every d
static const long long kNaDoubles = kNaMaxD + (long long)kNaMaxM * kNaFeatCh + kNaMaxM +
                                    (long long)kNaMaxP * kNaNnCh + kNaMaxP + RNP_MAX_M + 6;
static const long long kNaInts = 2 + RNP_MAX_M + 4;

static __device__ __align__(256) double g_na_scratch[kNaDoubles + (kNaInts + 1) / 2];

struct NaLayout {
  double *q, *feat_part, *phiq, *nn_part, *dist, *alpha, *sc, *sr;
  int *P, *meff, *idx, *flags;
};

static NaLayout layout(double* base) {
  NaLayout L;
  double* p = base;
  L.q = p; p += kNaMaxD;
  L.feat_part = p; p += (long long)kNaMaxM * kNaFeatCh;
  L.phiq = p; p += kNaMaxM;
  L.nn_part = p; p += (long long)kNaMaxP * kNaNnCh;
  L.dist = p; p += kNaMaxP;
  L.alpha = p; p += RNP_MAX_M;
  L.sc = p; p += 3;
  L.sr = p; p += 3;
  int* ip = reinterpret_cast<int*>(p);
  L.P = ip; ip += 1;
  L.meff = ip; ip += 1;
  L.idx = ip; ip += RNP_MAX_M;
  L.flags = ip;
  return L;
}

// Writes the per-call values into the scratch and clears what must start at
// zero (the flags), so no host-to-device copy is needed.
__global__ void k_na_prologue(int* P, int Pv, double* sc, double* sr, double c0, double c1,
                              double c2, double r0, double r1, double r2, int* flags) {
  *P = Pv;
  sc[0] = c0; sc[1] = c1; sc[2] = c2;
  sr[0] = r0; sr[1] = r1; sr[2] = r2;
  flags[0] = flags[1] = flags[2] = flags[3] = 0;
}

__global__ void k_na_epilogue(const int* flags, int* status) {
  *status = flags[1] ? RNP_ENONFINITE : (flags[2] ? RNP_ENONFINITE : RNP_OK);
}

// Device address of the scratch array on the current device (a host-side
// mention of g_na_scratch is only a stand-in).  Looked up on every call: the
// first lookup on a device loads the module there, later ones are a table
// read, and a lookup per call stays right if the device's context is reset
// and the module reloads elsewhere.
static cudaError_t scratch_for_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace rnp

using namespace rnp;

extern "C" rnp_status rnp_randnet_predict_noalloc(const rnp_problem* prob, const double* A,
                                                  const double* zeta, const double* S,
                                                  const double* Y, const double* Phi, int P,
                                                  const double* c, const double* r,
                                                  const double* q, double* out,
                                                  int* status, void* cuda_stream) {
  if (!prob || !A || !zeta || !q || !out || !c || !r || P < 0 ||
      (P > 0 && (!S || !Y || !Phi))) {
    set_global_error("rnp_randnet_predict_noalloc: NULL argument or P < 0");
    return RNP_EINVAL;
  }
  const Geom g = make_geom(*prob);
  if (g.kp < 0 || prob->M < 1 || prob->m < 1 || prob->m > RNP_MAX_M) {
    set_global_error("rnp_randnet_predict_noalloc: bad problem");
    return RNP_EINVAL;
  }
  if (g.d > kNaMaxD || P > kNaMaxP || prob->M > kNaMaxM) {
    set_global_error(
        "rnp_randnet_predict_noalloc: size beyond the fixed scratch (d <= 262144, "
        "P <= 4096, M <= 1024)");
    return RNP_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return RNP_ECUDA;
  }
  const NaLayout L = layout(base);
  const int ncomp = g.ncomp;
  k_na_prologue<<<1, 1, 0, st>>>(L.P, P, L.sc, L.sr, c[0], ncomp > 1 ? c[1] : 0.0,
                                 ncomp > 2 ? c[2] : 0.0, r[0], ncomp > 1 ? r[1] : 1.0,
                                 ncomp > 2 ? r[2] : 1.0, L.flags);
  count_launches(1);
  const long long d = g.d;
  const int M = prob->M;
  Rows qrow{nullptr, 0, d};
  if ((e = launch_scale_rows(g, q, qrow, nullptr, 1, L.sc, L.sr, L.q, nullptr, qrow, 1, nullptr,
                             st)) ||
      (e = launch_features64(A, zeta, M, d, L.q, qrow, 1, L.phiq, Rows{nullptr, 0, M},
                             L.feat_part, nullptr, st)) ||
      (e = launch_nn_partial(L.q, S, P, d, L.P, P, 1, L.nn_part, nullptr, st)) ||
      (e = launch_topm_ridge(L.nn_part, d, Phi, P, M, L.phiq, M, nullptr, 0,
                             nullptr, L.P, P, 1,
                             prob->m, prob->lambda, L.dist, L.alpha, L.idx, L.meff,
                             L.flags + 0, L.flags + 1, nullptr, st)) ||
      (e = launch_update(nullptr, 0, Y, P, d, L.alpha, L.idx, L.meff, out, d, nullptr, 0,
                         L.flags + 2, 1, nullptr, st))) {
    set_global_error(cudaGetErrorString(e));
    return RNP_ECUDA;
  }
  if (status) {
    k_na_epilogue<<<1, 1, 0, st>>>(L.flags, status);
    count_launches(1);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return RNP_ECUDA;
  }
  return RNP_OK;
}
