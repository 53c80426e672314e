// certificate.cu -- the second-order optimality test of Lemma 3.2 (Eq. sec-opt)
// on the GPU: the smallest value of grad^2 F(X)[D,D] - theta D^*D over unit D
// in the tangent set T_X = {D : X^*D = 0} (Eq. tangent-St), by Lanczos with
// full reorthogonalisation on the operator
//     K(d) = P (H''(psi) d - mu d),   P d = d - psi <psi, d>_h   (complex <.,.>)
// in grid units, where H''(psi) d is gpe_hessvec (Lemma 3.1) and mu the
// chemical potential; in the unified units of Eq. prob the quadratic form is
// twice that of K (X = sqrt(h_vol) psi, theta = 2 mu, grad^2 F = 2 sqrt(h_vol)
// H'' per unit), so the reported value is 2 lambda_min(K).
//
// Every vector operation runs on the device (the operator passes, the
// moment reductions, axpby); the host keeps the Lanczos tridiagonal and finds
// its smallest eigenvalue by Sturm-sequence bisection and its eigenvector by
// inverse iteration.
#include <math.h>
#include <string.h>
#include <algorithm>
#include <vector>
#include "ops_impl.cuh"

namespace gpe {

// y = i x (complex interleaved)
template <typename T>
__global__ void k_times_i(const void* xv, void* yv, long long n) {
  using C = typename C2t<T>::type;
  const C* x = (const C*)xv;
  C* y = (C*)yv;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const C v = x[k];
    C r;
    r.x = -v.y;
    r.y = v.x;
    y[k] = r;
  }
}

// part[i][b] = sum over block b's elements of Re(conj(V_i) w)   (i < n)
template <typename T, bool CPLX>
__global__ void __launch_bounds__(256) k_multidot(const void* Vv, long long M, int n, const void* wv, int nb,
                                                  double* part) {
  using V = typename VT<T, CPLX>::V;
  const int i = blockIdx.y;
  const V* v = (const V*)Vv + (size_t)i * M;
  const V* w = (const V*)wv;
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < M; e += (long long)nb * blockDim.x)
    acc += dre(v[e], w[e]);
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    part[(size_t)i * nb + blockIdx.x] = t;
  }
}

// out[i] = h * sum_b part[i][b] (fixed order)
__global__ void k_fold_rows(const double* part, int nb, int n, double h, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += part[(size_t)i * nb + b];
  out[i] = h * t;
}

// w -= sum_{i < n} c_i V_i   (c on the device)
template <typename T, bool CPLX>
__global__ void k_multi_axpy(const void* Vv, long long M, int n, const double* c, void* wv) {
  using V = typename VT<T, CPLX>::V;
  const V* v = (const V*)Vv;
  V* w = (V*)wv;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < M; e += (long long)gridDim.x * blockDim.x) {
    V a = w[e];
    for (int i = 0; i < n; ++i) a = a - (T)c[i] * v[(size_t)i * M + e];
    w[e] = a;
  }
}

namespace {

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x
// (Sturm sequence of the LDL^T pivots).
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, int n, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < n; ++i) {
    const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Smallest eigenvalue of the n x n symmetric tridiagonal by bisection.
double tri_min_eig(const std::vector<double>& a, const std::vector<double>& b, int n) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < n ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(1.0, fmax(fabs(lo), fabs(hi))); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, n, mid) >= 1) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Unit eigenvector of the tridiagonal for the eigenvalue lam: inverse
// iteration with a tiny shift, each solve by Gaussian elimination with partial
// pivoting on the tridiagonal (row interchanges create a second
// superdiagonal).
std::vector<double> tri_eigvec(const std::vector<double>& a, const std::vector<double>& b, int n, double lam) {
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(a[i]) + (i + 1 < n ? fabs(b[i]) : 0.0));
  const double sh = lam - 1e-12 * fmax(scale, 1.0);
  std::vector<double> y(n, 1.0);
  if (n == 1) return y;
  for (int it = 0; it < 3; ++it) {
    std::vector<double> dl(n - 1), d(n), du(n - 1), du2(n > 2 ? n - 2 : 1, 0.0), x = y;
    for (int i = 0; i < n; ++i) d[i] = a[i] - sh;
    for (int i = 0; i + 1 < n; ++i) dl[i] = du[i] = b[i];
    for (int i = 0; i + 1 < n; ++i) {
      if (fabs(d[i]) >= fabs(dl[i])) {
        if (d[i] == 0.0) d[i] = 1e-300;
        const double f = dl[i] / d[i];
        d[i + 1] -= f * du[i];
        x[i + 1] -= f * x[i];
        if (i + 2 < n) du2[i] = 0.0;
      } else {
        const double f = d[i] / dl[i];
        d[i] = dl[i];
        const double t = d[i + 1];
        d[i + 1] = du[i] - f * t;
        if (i + 2 < n) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du2[i];
        }
        du[i] = t;
        const double xt = x[i];
        x[i] = x[i + 1];
        x[i + 1] = xt - f * x[i + 1];
      }
    }
    if (d[n - 1] == 0.0) d[n - 1] = 1e-300;
    x[n - 1] /= d[n - 1];
    x[n - 2] = (x[n - 2] - du[n - 2] * x[n - 1]) / d[n - 2];
    for (int i = n - 3; i >= 0; --i) x[i] = (x[i] - du[i] * x[i + 1] - du2[i] * x[i + 2]) / d[i];
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm += x[i] * x[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < n; ++i) y[i] = x[i] / nrm;
  }
  return y;
}

}  // namespace

template <typename T>
struct CertWork {
  gpe_plan p;
  cudaStream_t st;
  long long M;
  int cplx;
  size_t vb;
  double hv;
  int cap = 0;                  // basis vectors held
  int nb = 0;                   // blocks per vector of the batched dot
  double* d_coef = nullptr;     // [cap + 2] coefficients / dot results
  double* d_part = nullptr;     // [cap][nb] partial dots
  double* h_buf = nullptr;      // [cap + 2] pinned
  void* Vb = nullptr;           // basis v_0 .. v_{cap-1}, contiguous
  void* w = nullptr;
  void* u = nullptr;
  void* ipsi = nullptr;
  ~CertWork() {
    cudaFree(Vb);
    cudaFree(w);
    cudaFree(u);
    cudaFree(ipsi);
    cudaFree(d_coef);
    cudaFree(d_part);
    cudaFreeHost(h_buf);
  }
  void* vec(int i) const { return (char*)Vb + (size_t)i * vb; }
  // out[i] = Re <v_i, x>_h for i < n (one batched reduction, fixed order)
  gpe_status dots(int n, const void* x, const void* vbase, double* out) {
    dim3 grid(nb, n);
    if (cplx) k_multidot<T, true><<<grid, 256, 0, st>>>(vbase, M, n, x, nb, d_part);
    else k_multidot<T, false><<<grid, 256, 0, st>>>(vbase, M, n, x, nb, d_part);
    GPE_CUDA(cudaGetLastError());
    k_fold_rows<<<(n + 127) / 128, 128, 0, st>>>(d_part, nb, n, hv, d_coef);
    GPE_CUDA(cudaGetLastError());
    GPE_CUDA(cudaMemcpyAsync(h_buf, d_coef, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    GPE_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) out[i] = h_buf[i];
    return GPE_OK;
  }
  gpe_status dot(const void* a, const void* x, double* out) { return dots(1, x, a, out); }
  // x -= sum_{i<n} c_i v_i  (c on the host)
  gpe_status combine(int n, const double* c, const void* vbase, void* x) {
    for (int i = 0; i < n; ++i) h_buf[i] = c[i];
    GPE_CUDA(cudaMemcpyAsync(d_coef, h_buf, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    const int g = (int)std::min<long long>((M + 255) / 256, 2048);
    if (cplx) k_multi_axpy<T, true><<<g, 256, 0, st>>>(vbase, M, n, d_coef, x);
    else k_multi_axpy<T, false><<<g, 256, 0, st>>>(vbase, M, n, d_coef, x);
    GPE_CUDA(cudaGetLastError());
    // the pinned coefficient buffer is reused by the next call
    GPE_CUDA(cudaStreamSynchronize(st));
    return GPE_OK;
  }
  gpe_status scale(void* x, double a) {
    const double c = 1.0 - a;   // x -= (1 - a) x
    return combine(1, &c, x, x);
  }
  // d <- P d: remove the components along psi and, for complex data, i psi
  gpe_status project(const void* psi, double n2, void* d) {
    double c;
    gpe_status s = dot(psi, d, &c);
    if (s == GPE_OK) {
      c /= n2;
      s = combine(1, &c, psi, d);
    }
    if (s == GPE_OK && cplx) {
      s = dot(ipsi, d, &c);
      if (s == GPE_OK) {
        c /= n2;
        s = combine(1, &c, ipsi, d);
      }
    }
    return s;
  }
};

template <typename T>
static gpe_status cert_impl(gpe_plan p, const void* psi, int max_iter, double tol, double* lambda, double* resid,
                            int* iters) {
  CertWork<T> W;
  W.p = p;
  W.st = p->stream;
  W.M = p->g.M;
  W.cplx = p->g.is_complex;
  W.vb = elem_size(p->prec, W.cplx) * (size_t)W.M;
  W.hv = p->g.hvol;
  W.cap = max_iter;
  W.nb = (int)std::max<long long>(1, std::min<long long>((W.M + 255) / 256, 64));
  double E = 0, mu = 0, n2 = 0;
  gpe_status s = gpe_energy(p, psi, &E, &mu, &n2);
  if (s != GPE_OK) return s;
  if (!(n2 > 0.0)) return fail(GPE_EINVAL, "psi is zero");
  GPE_CUDA(cudaMalloc(&W.Vb, W.vb * (size_t)W.cap));
  GPE_CUDA(cudaMalloc(&W.w, W.vb));
  GPE_CUDA(cudaMalloc(&W.u, W.vb));
  GPE_CUDA(cudaMalloc(&W.d_coef, sizeof(double) * (W.cap + 2)));
  GPE_CUDA(cudaMalloc(&W.d_part, sizeof(double) * (size_t)W.nb * (W.cap + 2)));
  GPE_CUDA(cudaMallocHost(&W.h_buf, sizeof(double) * (W.cap + 2)));
  if (W.cplx) {
    GPE_CUDA(cudaMalloc(&W.ipsi, W.vb));
    k_times_i<T><<<(int)std::min<long long>((W.M + 255) / 256, 4096), 256, 0, W.st>>>(psi, W.ipsi, W.M);
    GPE_CUDA(cudaGetLastError());
  }
  // deterministic pseudo-random start vector (xorshift64), projected onto T_X
  {
    const long long nr = W.M * (W.cplx ? 2 : 1);
    std::vector<T> h((size_t)nr);
    unsigned long long x = 0x9E3779B97F4A7C15ull;
    for (long long i = 0; i < nr; ++i) {
      x ^= x << 13;
      x ^= x >> 7;
      x ^= x << 17;
      h[(size_t)i] = (T)((double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
    GPE_CUDA(cudaMemcpyAsync(W.vec(0), h.data(), W.vb, cudaMemcpyHostToDevice, W.st));
    GPE_CUDA(cudaStreamSynchronize(W.st));
  }
  s = W.project(psi, n2, W.vec(0));
  double nv = 0.0;
  if (s == GPE_OK) s = W.dot(W.vec(0), W.vec(0), &nv);
  if (s == GPE_OK) s = W.scale(W.vec(0), 1.0 / sqrt(nv));
  if (s != GPE_OK) return s;

  std::vector<double> a, b, c((size_t)W.cap + 2);
  double theta = 0.0;
  int n = 0;
  for (int k = 0; k < max_iter; ++k) {
    n = k + 1;
    // w = P (H'' v_k - mu v_k), then orthogonal to v_0..v_k (two passes of
    // classical Gram-Schmidt; the first pass's v_k coefficient is alpha_k)
    s = gpe_hessvec(p, psi, W.vec(k), -mu, W.w);
    if (s == GPE_OK) s = W.project(psi, n2, W.w);
    if (s == GPE_OK) s = W.dots(n, W.w, W.Vb, c.data());
    if (s != GPE_OK) return s;
    a.push_back(c[k]);
    s = W.combine(n, c.data(), W.Vb, W.w);
    if (s == GPE_OK) s = W.dots(n, W.w, W.Vb, c.data());
    if (s == GPE_OK) s = W.combine(n, c.data(), W.Vb, W.w);
    // back onto T_X: rounding leaves components along psi that the
    // orthogonalisation does not remove, and once the Krylov space nears the
    // tangent space's dimension they grow and pull the Ritz values below it
    if (s == GPE_OK) s = W.project(psi, n2, W.w);
    double bb = 0.0;
    if (s == GPE_OK) s = W.dot(W.w, W.w, &bb);
    if (s != GPE_OK) return s;
    const double beta = sqrt(fmax(bb, 0.0));
    theta = tri_min_eig(a, b, n);
    const std::vector<double> y = tri_eigvec(a, b, n, theta);
    const double est = beta * fabs(y[n - 1]);
    if (est <= tol * fmax(1.0, fabs(theta)) || beta <= 1e-13 * fmax(1.0, fabs(theta)) || k + 1 == max_iter) break;
    b.push_back(beta);
    GPE_CUDA(cudaMemcpyAsync(W.vec(k + 1), W.w, W.vb, cudaMemcpyDeviceToDevice, W.st));
    s = W.scale(W.vec(k + 1), 1.0 / beta);
    if (s != GPE_OK) return s;
  }
  // Ritz vector u = sum y_i v_i and its true residual |K u - theta u|_h
  const std::vector<double> y = tri_eigvec(a, b, n, theta);
  for (int i = 0; i < n; ++i) c[i] = -y[i];
  GPE_CUDA(cudaMemsetAsync(W.u, 0, W.vb, W.st));
  s = W.combine(n, c.data(), W.Vb, W.u);
  if (s == GPE_OK) s = gpe_hessvec(p, psi, W.u, -mu, W.w);
  if (s == GPE_OK) s = W.project(psi, n2, W.w);
  double cu = theta;
  if (s == GPE_OK) s = W.combine(1, &cu, W.u, W.w);
  double rr = 0.0, uu = 1.0;
  if (s == GPE_OK) s = W.dot(W.w, W.w, &rr);
  if (s == GPE_OK) s = W.dot(W.u, W.u, &uu);
  if (s != GPE_OK) return s;
  // unified units of Eq. sec-opt: twice the grid-unit values
  *lambda = 2.0 * theta;
  if (resid) *resid = 2.0 * sqrt(fmax(rr, 0.0) / fmax(uu, 1e-300));
  if (iters) *iters = n;
  if (!isfinite(theta)) return fail(GPE_ENONFINITE, "non-finite certificate");
  return GPE_OK;
}

}  // namespace gpe

using namespace gpe;

extern "C" gpe_status gpe_hess_min_eig(gpe_plan plan, const void* psi, int max_iter, double tol, double* lambda_min,
                                       double* residual, int* iters) {
  if (!plan || !psi || !lambda_min) return fail(GPE_EINVAL, "NULL argument");
  if (plan->g.nbatch != 1) return fail(GPE_EINVAL, "gpe_hess_min_eig needs a plan with nbatch = 1");
  const long long dim = plan->g.M * (plan->g.is_complex ? 2 : 1) - (plan->g.is_complex ? 2 : 1);
  if (max_iter < 2 || max_iter > 1000) return fail(GPE_EINVAL, "max_iter must be in [2, 1000]");
  if (!(tol > 0.0)) return fail(GPE_EINVAL, "tol must be positive");
  if (max_iter > dim) max_iter = (int)dim;
  return plan->prec == GPE_F64 ? cert_impl<double>(plan, psi, max_iter, tol, lambda_min, residual, iters)
                               : cert_impl<float>(plan, psi, max_iter, tol, lambda_min, residual, iters);
}
