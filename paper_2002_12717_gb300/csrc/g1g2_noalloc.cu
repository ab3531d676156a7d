// g1g2_g1_rhs_noalloc: the G1 right-hand side for callers that must not
// allocate device memory.
//
// It computes the same dn/dt as the G1 part of g1g2_rhs (Hartree-Fock build,
// split-K collision integral, commutator), but its scratch -- the split-K
// partial sums of the collision integral, h^HF and I -- lives in one
// file-scope device array instead of context buffers, so a call allocates
// nothing.  The array exists once per GPU that loads the library and stays
// until the process exits.
#include "g1g2_internal.h"

#include <mutex>
#include <string>

namespace {

constexpr int kMaxNb = 64;       // largest basis accepted
constexpr int kMaxSplits = 32;   // split-K slices of the collision integral
constexpr size_t kScratchElems = (size_t)(kMaxSplits + 2) * kMaxNb * kMaxNb;  // 2.2 MB of double2

// One shared scratch area for every call on a device: [partials | hHF | I].
static __device__ __align__(256) double2 g_noalloc_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
// Address of the array on each device; only a successful lookup is kept, so a
// first call that failed for a passing reason (say, inside a stream capture)
// does not block later calls on that device.
double2 *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// h^HF_ij = h_ij + sum_kl (w_ikjl - w_iklj) n_lk  (restricted: no exchange term), w in the ABI layout.
__global__ void hf_from_abi_w_kernel(int nb, int restricted, const double2 *__restrict__ h,
                                     const double2 *__restrict__ w, const double2 *__restrict__ n,
                                     double2 *__restrict__ hhf) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nb * nb) return;
  const int i = warp / nb, j = warp % nb;
  const long long N = nb;
  double2 acc = {0.0, 0.0};
  for (int c = lane; c < nb * nb; c += 32) {
    const int k = c / nb, l = c % nb;
    double2 a = w[((i * N + k) * N + j) * N + l];
    if (!restricted) {
      const double2 b = w[((i * N + k) * N + l) * N + j];
      a.x -= b.x;
      a.y -= b.y;
    }
    const double2 v = n[l * N + k];
    acc.x = fma(a.x, v.x, fma(-a.y, v.y, acc.x));
    acc.y = fma(a.x, v.y, fma(a.y, v.x, acc.y));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) hhf[warp] = {h[warp].x + acc.x, h[warp].y + acc.y};
}

// Device address of the scratch array on the current device: looked up with that
// device current until one lookup succeeds, then reused.
cudaError_t scratch_on_current_device(double2 **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();  // the failed lookup leaves no pending error behind
      return e;
    }
    g_scratch_ptr[dev] = static_cast<double2 *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int g1g2_g1_rhs_noalloc(int nb, int restricted, const double *h_dev, const double *w_dev,
                                   const double *n_dev, const double *G2_dev, double *dn_dev, void *cuda_stream) {
  using namespace g1g2;
  if (nb < 1 || nb > kMaxNb) {
    g1g2::set_error_detail("nb = " + std::to_string(nb) + " is outside [1, " + std::to_string(kMaxNb) +
                           "], the size of the no-allocation scratch");
    return G1G2_EINVAL;
  }
  if (!h_dev || !w_dev || !n_dev || !G2_dev || !dn_dev) {
    g1g2::set_error_detail("NULL device pointer");
    return G1G2_EINVAL;
  }
  // A non-sticky error left pending by unrelated earlier work would otherwise be
  // picked up by the launch checks below and reported as this call's failure.
  cudaGetLastError();
  double2 *scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) {
    g1g2::set_error_detail(std::string("scratch lookup failed: ") + cudaGetErrorString(e));
    return G1G2_ECUDA;
  }
  const long long N = nb, N2 = N * N;
  double2 *partial = scratch;                      // kMaxSplits * nb^2
  double2 *hhf = scratch + (size_t)kMaxSplits * N2;
  double2 *I = hhf + N2;
  const cplx *h = reinterpret_cast<const cplx *>(h_dev);
  const cplx *w = reinterpret_cast<const cplx *>(w_dev);
  const cplx *n = reinterpret_cast<const cplx *>(n_dev);
  const cplx *G = reinterpret_cast<const cplx *>(G2_dev);

  Launcher L;
  L.stream = static_cast<cudaStream_t>(cuda_stream);
  const int blocks = (int)((N2 * 32 + 255) / 256);
  hf_from_abi_w_kernel<<<blocks, 256, 0, L.stream>>>(nb, restricted, h, w, n, hhf);
  L.after_launch();
  // I_ij = -i sum_k sum_(lp) w[i][k][(lp)] G[(lp)][j][k]: batches over k, reduced over the splits.
  ZGemm g;
  g.M = nb; g.N = nb; g.K = (int)N2; g.batch = nb;
  g.A = w; g.sa_b = N2; g.sa_m = N2 * N; g.sa_k = 1;
  g.B = G; g.sb_b = 1; g.sb_k = N2; g.sb_n = N;
  g.C = I; g.sc_m = N; g.sc_n = 1;
  g.alpha = {0.0, -1.0};
  zgemm_reduce(L, g, partial, kMaxSplits);
  Rk4Stage st{-1, 0.0};
  g1_update(L, nb, hhf, n, I, st, nullptr, nullptr, nullptr, reinterpret_cast<cplx *>(dn_dev));
  if (L.err != cudaSuccess) {
    g1g2::set_error_detail(std::string("launch failed: ") + cudaGetErrorString(L.err));
    return G1G2_ECUDA;
  }
  return G1G2_OK;
}
