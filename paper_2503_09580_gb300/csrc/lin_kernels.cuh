// Kernels of the generic (FP64 / FP32) path of Algorithm 1.
//
// A batched 3-D real transform is split into
//   * plane kernels: for each i1-plane, the axis-3 real<->half-complex
//     transform (two real rows packed into one complex row) and the axis-2
//     complex transform, done in shared memory;
//   * axis-1 kernels: for a tile of (p2, k3) columns of one instance, the
//     axis-1 complex transform, fused with the pointwise stage that follows
//     it (a product with r^, a multiplier table indexed by |k|^2, or the
//     accumulation of phi_j psi^_j into L^+).
// Half-spectrum layout per instance: [p1][p2][k3], k3 = 0..N/2 natural,
// p1, p2 digit-reversed positions (see fft.cuh); H = N*N*(N/2+1).
// Real fields: [i1][i2][i3] centred order (v_i = (i - N/2) h), except the
// kernel u_j = M^g phit_j, which is indexed by cyclic displacement.
#pragma once
#include "fft.cuh"

namespace lbo {

struct InstanceParams {
  double rho, u1, u2, u3, theta;
};

__device__ __forceinline__ InstanceParams load_params(const double* p, int b) {
  InstanceParams q;
  q.rho = p[5 * b + 0];
  q.u1 = p[5 * b + 1];
  q.u2 = p[5 * b + 2];
  q.u3 = p[5 * b + 3];
  q.theta = p[5 * b + 4];
  return q;
}

// Sources of the real plane fed to a forward plane transform.
enum PlaneSrc {
  SRC_RATIO = 0,   // r = g / M, 0 where the cut-off of Eq. (3.9) applies
  SRC_REAL64 = 1,  // a double field (the ABI input g)
  SRC_MAXW = 2,    // the Maxwellian M
  SRC_REALT = 4    // a field of the transform precision T (a.src)
};

struct PlaneArgs {
  const double* params;  // [B][5]
  const double* g;       // [B][N^3] (SRC_RATIO / SRC_REAL64)
  const void* src;       // [B][N^3] of T (SRC_REALT)
  double h;              // grid spacing
  double log_inv_eps;    // ln(1/eps)
  int cutoff;            // apply Eq. (3.9)
};

// Cut-off test of Eq. (3.9), M/rho < eps  <=>
//   |v-u|^2/(2 theta) > ln(1/eps) - 1.5 ln(2 pi theta).
// Every operation is rounded separately (no FMA contraction) so that the
// decision is reproducible.
__device__ __forceinline__ bool cut_point(double d2, double theta, double log_inv_eps) {
  double lhs = __ddiv_rn(d2, __dmul_rn(2.0, theta));
  double thr = __dsub_rn(log_inv_eps, __dmul_rn(1.5, log(__dmul_rn(__dmul_rn(2.0, 3.141592653589793), theta))));
  return lhs > thr;
}

__device__ __forceinline__ double sq_rn(double a) { return __dmul_rn(a, a); }

// |v - u|^2 at centred index (i1, i2, i3), as ((d1^2 + d2^2) + d3^2).
__device__ __forceinline__ double dist2(int i1, int i2, int i3, int N, double h, const InstanceParams& q) {
  double v1 = __dmul_rn((double)(i1 - N / 2), h), v2 = __dmul_rn((double)(i2 - N / 2), h),
         v3 = __dmul_rn((double)(i3 - N / 2), h);
  return __dadd_rn(__dadd_rn(sq_rn(__dsub_rn(v1, q.u1)), sq_rn(__dsub_rn(v2, q.u2))), sq_rn(__dsub_rn(v3, q.u3)));
}

__device__ __forceinline__ double maxwellian(double d2, const InstanceParams& q) {
  return q.rho * pow(2.0 * 3.141592653589793 * q.theta, -1.5) * exp(-d2 / (2.0 * q.theta));
}

// Per-instance separable Maxwellian tables, filled once per CTA:
//   em[d*N + i] = exp(-(v_i - u_d)^2 / (2 theta)), axis 0 times the
//   prefactor rho (2 pi theta)^{-3/2}, so M(v) = em[i1] em[N+i2] em[2N+i3];
//   *thr = ln(1/eps) - 1.5 ln(2 pi theta), the cut-off threshold of Eq. (3.9).
template <int N>
__device__ __forceinline__ void fill_maxwellian_tables(double* em, double* thr, const InstanceParams& q, double h,
                                                       double log_inv_eps) {
  for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) {
    int d = t / N, i = t % N;
    double ud = d == 0 ? q.u1 : (d == 1 ? q.u2 : q.u3);
    double v = (double)(i - N / 2) * h - ud;
    double e = exp(-(v * v) / (2.0 * q.theta));
    if (d == 0) e *= q.rho * pow(2.0 * 3.141592653589793 * q.theta, -1.5);
    em[t] = e;
  }
  if (threadIdx.x == 0)
    *thr = __dsub_rn(log_inv_eps, __dmul_rn(1.5, log(__dmul_rn(__dmul_rn(2.0, 3.141592653589793), q.theta))));
  __syncthreads();
}

// Tables of the ratio source r = g/M, filled once per CTA:
//   ei[d*N + i] = exp(+(v_i - u_d)^2 / (2 theta)), axis 0 divided by the
//   prefactor rho (2 pi theta)^{-3/2}, so 1/M = ei[i1] ei[N+i2] ei[2N+i3];
//   *dstar = the smallest |v-u|^2 for which fl(|v-u|^2 / (2 theta)) > thr,
//   thr = ln(1/eps) - 1.5 ln(2 pi theta).  The cut-off test of Eq. (3.9) is
//   monotone in |v-u|^2, so |v-u|^2 >= dstar takes exactly the same
//   decision as the oracle's division, point by point, without dividing.
template <int N>
__device__ __forceinline__ void fill_ratio_tables(double* ei, double* dstar, const InstanceParams& q, double h,
                                                  double log_inv_eps) {
  for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) {
    const int d = t / N, i = t % N;
    const double ud = d == 0 ? q.u1 : (d == 1 ? q.u2 : q.u3);
    const double dv = __dsub_rn(__dmul_rn((double)(i - N / 2), h), ud);
    double e = exp(__dmul_rn(dv, dv) / (2.0 * q.theta));
    if (d == 0) e /= q.rho * pow(2.0 * 3.141592653589793 * q.theta, -1.5);
    ei[t] = e;
  }
  if (threadIdx.x == 0) {
    const double twoth = __dmul_rn(2.0, q.theta);
    const double thr = __dsub_rn(log_inv_eps, __dmul_rn(1.5, log(__dmul_rn(__dmul_rn(2.0, 3.141592653589793), q.theta))));
    double x = __dmul_rn(thr, twoth);
    for (int it = 0; it < 64 && __ddiv_rn(x, twoth) > thr; ++it) x = nextafter(x, -1e308);
    for (int it = 0; it < 64 && !(__ddiv_rn(x, twoth) > thr); ++it) x = nextafter(x, 1e308);
    *dstar = x;
  }
  __syncthreads();
}

// The source fields of the forward plane transforms.  For SRC_MAXW, em and
// thr are the tables of fill_maxwellian_tables; for SRC_RATIO, those of
// fill_ratio_tables (em = the reciprocal factors, thr = dstar).
template <typename T, int N, int SRC>
__device__ __forceinline__ T plane_source(const PlaneArgs& a, const InstanceParams& q, int b, int i1, int i2, int i3,
                                          const double* em, double thr) {
  size_t idx = (((size_t)b * N + i1) * N + i2) * N + i3;
  if constexpr (SRC == SRC_REALT) {
    return ((const T*)a.src)[idx];
  } else if constexpr (SRC == SRC_REAL64) {
    return (T)a.g[idx];
  } else if constexpr (SRC == SRC_MAXW) {
    return (T)(em[i1] * em[N + i2] * em[2 * N + i3]);
  } else {  // SRC_RATIO: r = g / M, 0 where the cut-off of Eq. (3.9) applies
    if (a.cutoff && dist2(i1, i2, i3, N, a.h, q) >= thr) return (T)0;
    return (T)(a.g[idx] * ((em[i1] * em[N + i2]) * em[2 * N + i3]));
  }
}

// ------------------------------------------------------------ plane parts
// Shared memory of a plane kernel handling PPC planes:
//   A: [PPC][N/2][N]  packed complex rows along i3  (pencil ps=N, es=1)
//   B: [N][PPC][N/2+1] half rows; axis-2 pencils p = pp*(N/2+1)+k3,
//      ps = 1, es = PPC*(N/2+1)
template <typename T, int N, int PPC>
struct PlaneSmem {
  static constexpr int HC = N / 2 + 1;
  static constexpr int A_ELEMS = PPC * (N / 2) * N;
  static constexpr int B_ELEMS = N * PPC * HC;
  static constexpr size_t BYTES = sizeof(cpx<T>) * (A_ELEMS + B_ELEMS);
};

// A (packed rows, after the forward i3 transform) -> B half rows, then the
// forward axis-2 transform of B.
template <typename T, int N, int PPC>
__device__ __forceinline__ void plane_forward_from_A(cpx<T>* A, cpx<T>* B) {
  constexpr int HC = N / 2 + 1;
  smem_fft<T, N, false, false>(A, PPC * (N / 2), N, 1);
  for (int t = threadIdx.x; t < PPC * (N / 2) * HC; t += blockDim.x) {
    int k3 = t % HC, rest = t / HC, qq = rest % (N / 2), pp = rest / (N / 2);
    const cpx<T>* z = A + (pp * (N / 2) + qq) * N;
    cpx<T> z1 = z[pos_of_freq<N>(k3)], z2 = conjc(z[pos_of_freq<N>((N - k3) % N)]);
    cpx<T> xa = cscale(z1 + z2, (T)0.5);
    cpx<T> d = z1 - z2;
    cpx<T> xb = make_c((T)0.5 * d.y, (T)-0.5 * d.x);  // (z1 - conj z2) / (2i)
    B[((2 * qq) * PPC + pp) * HC + k3] = xa;
    B[((2 * qq + 1) * PPC + pp) * HC + k3] = xb;
  }
  __syncthreads();
  smem_fft<T, N, false, true>(B, PPC * HC, 1, PPC * HC);
}

// B (half spectrum, axis 2 in digit-reversed positions) -> inverse axis 2 ->
// packed rows in A -> inverse i3 transform: A[pp][q][i3] = x[2q][i3] + i x[2q+1][i3].
template <typename T, int N, int PPC>
__device__ __forceinline__ void plane_inverse_to_A(cpx<T>* A, cpx<T>* B) {
  constexpr int HC = N / 2 + 1;
  smem_fft<T, N, true, true>(B, PPC * HC, 1, PPC * HC);
  for (int t = threadIdx.x; t < PPC * (N / 2) * N; t += blockDim.x) {
    int k3 = t % N, rest = t / N, qq = rest % (N / 2), pp = rest / (N / 2);
    const cpx<T>* ra = B + ((2 * qq) * PPC + pp) * HC;
    const cpx<T>* rb = B + ((2 * qq + 1) * PPC + pp) * HC;
    cpx<T> xa, xb;
    if (k3 == 0 || k3 == N / 2) {
      xa = make_c(ra[k3].x, (T)0);
      xb = make_c(rb[k3].x, (T)0);
    } else if (k3 < N / 2) {
      xa = ra[k3];
      xb = rb[k3];
    } else {
      xa = conjc(ra[N - k3]);
      xb = conjc(rb[N - k3]);
    }
    A[(pp * (N / 2) + qq) * N + pos_of_freq<N>(k3)] = make_c(xa.x - xb.y, xa.y + xb.x);  // xa + i xb
  }
  __syncthreads();
  smem_fft<T, N, true, false>(A, PPC * (N / 2), N, 1);
}

template <typename T, int N, int PPC>
__device__ __forceinline__ void plane_store_B(const cpx<T>* B, cpx<T>* dst, int b, int i1_0) {
  constexpr int HC = N / 2 + 1;
  for (int t = threadIdx.x; t < PPC * N * HC; t += blockDim.x) {
    int k3 = t % HC, rest = t / HC, k2 = rest % N, pp = rest / N;
    dst[(((size_t)b * N + i1_0 + pp) * N + k2) * HC + k3] = B[(k2 * PPC + pp) * HC + k3];
  }
}

template <typename T, int N, int PPC>
__device__ __forceinline__ void plane_load_B(cpx<T>* B, const cpx<T>* src, int b, int i1_0) {
  constexpr int HC = N / 2 + 1;
  for (int t = threadIdx.x; t < PPC * N * HC; t += blockDim.x) {
    int k3 = t % HC, rest = t / HC, k2 = rest % N, pp = rest / N;
    B[(k2 * PPC + pp) * HC + k3] = src[(((size_t)b * N + i1_0 + pp) * N + k2) * HC + k3];
  }
  __syncthreads();
}

// Per-instance separable tables for M^h = rho (pi theta)^{-3/2} prod_d exp(-(v_d-u_d)^2/theta):
// eh[d*N + i] = exp(-(v_i-u_d)^2/theta), axis 1 carries the prefactor.
template <int N>
__device__ __forceinline__ void fill_mh_tables(double* eh, const InstanceParams& q, double h) {
  for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) {
    int d = t / N, i = t % N;
    double ud = d == 0 ? q.u1 : (d == 1 ? q.u2 : q.u3);
    double v = (double)(i - N / 2) * h - ud;
    double e = exp(-(v * v) / q.theta);
    if (d == 0) e *= q.rho * pow(3.141592653589793 * q.theta, -1.5);
    eh[t] = e;
  }
  __syncthreads();
}

// Forward plane transform of a real source field -> half spectrum (axis 1
// untransformed).  grid = (N/PPC, B).
template <typename T, int N, int PPC, int SRC>
__global__ void __launch_bounds__(256) k_plane_fwd(PlaneArgs a, cpx<T>* __restrict__ dst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* A = (cpx<T>*)smem_raw;
  cpx<T>* B = A + PlaneSmem<T, N, PPC>::A_ELEMS;
  __shared__ double em[3 * N];
  __shared__ double thr;
  const int b = blockIdx.y, i1_0 = blockIdx.x * PPC;
  const InstanceParams q = load_params(a.params, b);
  if constexpr (SRC == SRC_RATIO) fill_ratio_tables<N>(em, &thr, q, a.h, a.log_inv_eps);
  else if constexpr (SRC == SRC_MAXW) fill_maxwellian_tables<N>(em, &thr, q, a.h, a.log_inv_eps);
  for (int t = threadIdx.x; t < PPC * (N / 2) * N; t += blockDim.x) {
    int i3 = t % N, rest = t / N, qq = rest % (N / 2), pp = rest / (N / 2);
    int i1 = i1_0 + pp;
    T x0 = plane_source<T, N, SRC>(a, q, b, i1, 2 * qq, i3, em, thr);
    T x1 = plane_source<T, N, SRC>(a, q, b, i1, 2 * qq + 1, i3, em, thr);
    A[(pp * (N / 2) + qq) * N + i3] = make_c(x0, x1);
  }
  __syncthreads();
  plane_forward_from_A<T, N, PPC>(A, B);
  plane_store_B<T, N, PPC>(B, dst, b, i1_0);
}

enum PlaneInvMode {
  INV_TO_REAL = 0,    // write the real field (T) to dst_real
  INV_MH_FWD = 1      // multiply by M^h and transform forward again, in place
};

template <typename T, int N, int PPC, int MODE>
__global__ void __launch_bounds__(256) k_plane_inv(PlaneArgs a, cpx<T>* __restrict__ src, T* __restrict__ dst_real) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* A = (cpx<T>*)smem_raw;
  cpx<T>* B = A + PlaneSmem<T, N, PPC>::A_ELEMS;
  __shared__ double eh[3 * N];
  __shared__ T ehT[is_twofold<T>::value ? 3 * N : 1];  // eh in T: the two-fold forms stay on their pipe
  const int b = blockIdx.y, i1_0 = blockIdx.x * PPC;
  const InstanceParams q = load_params(a.params, b);
  if constexpr (MODE == INV_MH_FWD) {
    fill_mh_tables<N>(eh, q, a.h);
    if constexpr (is_twofold<T>::value) {
      for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) ehT[t] = T(eh[t]);
    }
  }
  plane_load_B<T, N, PPC>(B, src, b, i1_0);
  plane_inverse_to_A<T, N, PPC>(A, B);
  if constexpr (MODE == INV_TO_REAL) {
    for (int t = threadIdx.x; t < PPC * (N / 2) * N; t += blockDim.x) {
      int i3 = t % N, rest = t / N, qq = rest % (N / 2), pp = rest / (N / 2);
      cpx<T> z = A[(pp * (N / 2) + qq) * N + i3];
      size_t o = (((size_t)b * N + i1_0 + pp) * N + 2 * qq) * N + i3;
      dst_real[o] = z.x;
      dst_real[o + N] = z.y;
    }
  } else {
    for (int t = threadIdx.x; t < PPC * (N / 2) * N; t += blockDim.x) {
      int i3 = t % N, rest = t / N, qq = rest % (N / 2), pp = rest / (N / 2);
      int i1 = i1_0 + pp;
      cpx<T>& z = A[(pp * (N / 2) + qq) * N + i3];
      if constexpr (is_twofold<T>::value) {
        const T m13 = ehT[i1] * ehT[2 * N + i3];
        z.x = z.x * (m13 * ehT[N + 2 * qq]);
        z.y = z.y * (m13 * ehT[N + 2 * qq + 1]);
      } else {
        double m13 = eh[i1] * eh[2 * N + i3];
        z.x = (T)((double)z.x * (m13 * eh[N + 2 * qq]));
        z.y = (T)((double)z.y * (m13 * eh[N + 2 * qq + 1]));
      }
    }
    __syncthreads();
    plane_forward_from_A<T, N, PPC>(A, B);
    plane_store_B<T, N, PPC>(B, src, b, i1_0);
  }
}

// ------------------------------------------------------------ axis 1
enum Axis1Mode {
  AX_FWD_STORE = 0,   // dst = F1(src)
  AX_FWD_MULT_INV = 2,// dst = F1^-1( F1(src) * table[|k|^2] )
  AX_FWD_ACC = 3,     // dst (+)= table[|k|^2] * F1(src)
  AX_INV_STORE = 4,   // dst = F1^-1(src)
  AX_UHAT_INV = 5,    // dst = F1^-1( src * u^_j(|k|) * scale ), src already axis-1 transformed;
                      // u^_j from its axes-3,2 DCT planes, finished along axis 1 here
  AX_UHAT_CACHED = 6, // as AX_UHAT_INV with u^_j read whole from its cached octant
  AX_FWD_MULT3_INV = 7 // dst = F1^-1( F1(src) * table3[position] ), a multiplier per half-spectrum
                       // position ([N][N][N/2+1], the spectrum's own layout)
};

struct Axis1Args {
  const void* table;    // [QMAX] T (AX_FWD_MULT_INV, AX_FWD_ACC)
  double scale;         // AX_UHAT_INV, AX_UHAT_CACHED
  int first;            // AX_FWD_ACC: store instead of accumulate
  const void* uplanes;  // [B][N/2+1]^3 T: u^_j after the axis-3 and axis-2 DCTs (AX_UHAT_INV), or
                        // the whole octant u^_j(|k1|, |k2|, k3) (AX_UHAT_CACHED)
  const void* dct;      // [N/2+1][N/4] T (AX_UHAT_INV): DCT-I coefficients
};

// ------------------------------------------------------------ u^_j as a DCT-I
// u_j = M^g phit_j depends on the cyclic displacement d only through |d|, so
// it is real and even in each component of d, and its DFT u^_j is real and
// even in each component of k.  On the N-point cyclic grid that DFT is the
// separable DCT-I of length N/2 + 1 of the octant d in [0, N/2]^3:
//   U(k) = sum_d c_d x_d cos(2 pi k d / N),  c_0 = c_(N/2) = 1, c_d = 2 otherwise.
// Pairing d with N/2 - d (cos(2 pi k (N/2 - d) / N) = (-1)^k cos(2 pi k d / N))
// leaves N/4 terms per output: even k over x_d + x_(N/2-d) plus the middle
// term 2 x_(N/4) cos(pi k / 2), odd k over x_d - x_(N/2-d).
// dct[k * (N/4) + d] = c_d cos(2 pi k d / N), k = 0..N/2, d = 0..N/4-1.
template <typename T, int N>
struct DctPencil {
  static constexpr int HN = N / 2 + 1, Q4 = N / 4;
  T ev[Q4], od[Q4], mid;
  // x_d = src[d * stride], d = 0..N/2
  __device__ __forceinline__ void load(const T* src, size_t stride) {
#pragma unroll
    for (int d = 0; d < Q4; ++d) {
      const T a = src[d * stride], b = src[(N / 2 - d) * stride];
      ev[d] = a + b;
      od[d] = a - b;
    }
    mid = src[Q4 * stride];
  }
  __device__ __forceinline__ T out(int k, const T* dct) const {
    T acc;
    if (k & 1) {
      acc = (T)0;
#pragma unroll
      for (int d = 0; d < Q4; ++d) acc += dct[k * Q4 + d] * od[d];
    } else {
      acc = (k & 2) ? (T)-2 * mid : (T)2 * mid;
#pragma unroll
      for (int d = 0; d < Q4; ++d) acc += dct[k * Q4 + d] * ev[d];
    }
    return acc;
  }
};

// Octant planes per block of k_uhat_planes: at most 256 / (N/2+1) (one
// pencil per thread), spread evenly over the fewest blocks.
template <int N>
struct UhatPlanes {
  static constexpr int HC = N / 2 + 1;
  static constexpr int MAXP = (256 / HC) < HC ? (256 / HC) : HC;
  static constexpr int BLOCKS = (HC + MAXP - 1) / MAXP;
  static constexpr int PL = (HC + BLOCKS - 1) / BLOCKS;
};

// Axes 3 and 2 of u^_j for a block of PL octant planes d1 of one instance:
// w(d) = rho (pi theta)^-3/2 exp(-|d h|^2 / theta) phit_j(d), DCT-I along d3
// then d2, stored as up[b][d1][k2][k3].  grid = (ceil((N/2+1)/PL), B).
template <typename T, int N, int PL>
__global__ void __launch_bounds__(256) k_uhat_planes(const double* __restrict__ params, const T* __restrict__ phit,
                                                     const T* __restrict__ dct, double h, T* __restrict__ up) {
  constexpr int HN = N / 2 + 1, Q4 = N / 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* W = (T*)smem_raw;            // [PL][HN][HN]
  T* tab = W + PL * HN * HN;      // [HN][Q4]
  __shared__ double mg[HN + 1];   // mg[HN] = rho (pi theta)^-3/2
  __shared__ T mgT[is_twofold<T>::value ? HN + 1 : 1];
  const int b = blockIdx.y, d1_0 = blockIdx.x * PL;
  const int np = HN - d1_0 < PL ? HN - d1_0 : PL;
  const double rho = params[5 * b], theta = params[5 * b + 4];
  for (int t = threadIdx.x; t <= HN; t += blockDim.x) {
    if (t < HN) {
      const double x = t * h;
      mg[t] = exp(-(x * x) / theta);
    } else {
      mg[HN] = rho * pow(3.141592653589793 * theta, -1.5);
    }
  }
  for (int t = threadIdx.x; t < HN * Q4; t += blockDim.x) tab[t] = dct[t];
  __syncthreads();
  if constexpr (is_twofold<T>::value) {
    for (int t = threadIdx.x; t <= HN; t += blockDim.x) mgT[t] = T(mg[t]);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < np * HN * HN; t += blockDim.x) {
    const int d3 = t % HN, d2 = (t / HN) % HN, p = t / (HN * HN), d1 = d1_0 + p;
    if constexpr (is_twofold<T>::value) {
      W[t] = (mgT[HN] * (mgT[d1] * mgT[d2]) * mgT[d3]) * phit[((size_t)d1 * N + d2) * N + d3];
    } else {
      const double w = mg[HN] * (mg[d1] * mg[d2]) * mg[d3];
      W[t] = (T)(w * (double)phit[((size_t)d1 * N + d2) * N + d3]);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < np * HN; t += blockDim.x) {  // axis 3: pencil (p, d2)
    T* x = W + t * HN;
    DctPencil<T, N> pen;
    pen.load(x, 1);
    for (int k = 0; k < HN; ++k) x[k] = pen.out(k, tab);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < np * HN; t += blockDim.x) {  // axis 2: pencil (p, k3)
    T* x = W + (t / HN) * HN * HN + t % HN;
    DctPencil<T, N> pen;
    pen.load(x, HN);
    for (int k = 0; k < HN; ++k) x[k * HN] = pen.out(k, tab);
  }
  __syncthreads();
  T* dst = up + ((size_t)b * HN + d1_0) * HN * HN;
  for (int t = threadIdx.x; t < np * HN * HN; t += blockDim.x) dst[t] = W[t];
}

// Axis 1 of u^_j in place on the octant of k_uhat_planes, for the cache of
// the Maxwellian-dependent factors: up[b][d1][k2][k3] -> up[b][k1][k2][k3].
// Each thread reads one whole pencil before writing it, so in place is safe.
// grid = B.
template <typename T, int N>
__global__ void __launch_bounds__(256) k_uhat_finish(T* __restrict__ up, const T* __restrict__ dct) {
  constexpr int HN = N / 2 + 1;
  T* base = up + (size_t)blockIdx.x * HN * HN * HN;
  for (int t = threadIdx.x; t < HN * HN; t += blockDim.x) {
    T* x = base + t;  // pencil (k2, k3) = (t / HN, t % HN), stride HN^2 along axis 1
    DctPencil<T, N> pen;
    pen.load(x, (size_t)HN * HN);
    for (int k = 0; k < HN; ++k) x[(size_t)k * HN * HN] = pen.out(k, dct);
  }
}

template <typename T, int N, int CW, int MODE>
__global__ void __launch_bounds__(256) k_axis1(Axis1Args a, const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst) {
  constexpr int HC = N / 2 + 1, NC = N * HC;
  __shared__ __align__(16) cpx<T> S[N * CW];
  constexpr bool UHAT = MODE == AX_UHAT_INV || MODE == AX_UHAT_CACHED;
  __shared__ T Uc[UHAT ? CW * HC : 1];  // u^_j(|k1|, column)
  const int b = blockIdx.y, c0 = blockIdx.x * CW;
  const size_t inst = (size_t)b * N * NC;
  for (int t = threadIdx.x; t < N * CW; t += blockDim.x) {
    int c = t % CW, r = t / CW;
    S[t] = (c0 + c < NC) ? src[inst + (size_t)r * NC + c0 + c] : make_c((T)0, (T)0);
  }
  if constexpr (UHAT) {
    const T* up = (const T*)a.uplanes + (size_t)b * HC * HC * HC;
    if constexpr (MODE == AX_UHAT_INV) {
      // finish u^_j along axis 1 for this tile's columns (|k2|, k3): 8 threads
      // per column, each forming every 8th output
      const T* dct = (const T*)a.dct;
      for (int t = threadIdx.x; t < CW * 8; t += blockDim.x) {
        const int c = t % CW, gsub = t / CW, col = c0 + c;
        if (col >= NC) continue;
        const int p2 = col / HC, k3 = col % HC;
        int k2 = centred<N>(freq_of_pos<N>(p2));
        k2 = k2 < 0 ? -k2 : k2;
        DctPencil<T, N> pen;
        pen.load(up + (size_t)k2 * HC + k3, (size_t)HC * HC);
        for (int k = gsub; k < HC; k += 8) Uc[c * HC + k] = pen.out(k, dct);
      }
    } else {
      // the cached octant: u^_j(|k1|, |k2|, k3) at up[(|k1| HC + |k2|) HC + k3]
      for (int t = threadIdx.x; t < CW * HC; t += blockDim.x) {
        const int c = t % CW, k = t / CW, col = c0 + c;
        if (col >= NC) continue;
        const int p2 = col / HC, k3 = col % HC;
        int k2 = centred<N>(freq_of_pos<N>(p2));
        k2 = k2 < 0 ? -k2 : k2;
        Uc[c * HC + k] = up[((size_t)k * HC + k2) * HC + k3];
      }
    }
    __syncthreads();
    const T sc = (T)a.scale;
    for (int t = threadIdx.x; t < N * CW; t += blockDim.x) {
      int c = t % CW, r = t / CW;
      if (c0 + c < NC) {
        int k1 = centred<N>(freq_of_pos<N>(r));
        k1 = k1 < 0 ? -k1 : k1;
        S[t] = cscale(S[t], (T)(Uc[c * HC + k1] * sc));
      }
    }
    __syncthreads();
    smem_fft<T, N, true, true>(S, CW, 1, CW);
  } else {
    __syncthreads();
    if constexpr (MODE != AX_INV_STORE) smem_fft<T, N, false, true>(S, CW, 1, CW);
    else smem_fft<T, N, true, true>(S, CW, 1, CW);
  }
  if constexpr (MODE == AX_FWD_MULT_INV) {
    for (int t = threadIdx.x; t < N * CW; t += blockDim.x) {
      int c = t % CW, r = t / CW;
      if (c0 + c < NC) {
        int col = c0 + c, p2 = col / HC, k3 = col % HC;
        int k1 = centred<N>(freq_of_pos<N>(r)), k2 = centred<N>(freq_of_pos<N>(p2));
        S[t] = cscale(S[t], ((const T*)a.table)[k1 * k1 + k2 * k2 + k3 * k3]);
      }
    }
    __syncthreads();
    smem_fft<T, N, true, true>(S, CW, 1, CW);
  } else if constexpr (MODE == AX_FWD_MULT3_INV) {
    for (int t = threadIdx.x; t < N * CW; t += blockDim.x) {
      int c = t % CW, r = t / CW;
      if (c0 + c < NC) S[t] = cscale(S[t], ((const T*)a.table)[(size_t)r * NC + c0 + c]);
    }
    __syncthreads();
    smem_fft<T, N, true, true>(S, CW, 1, CW);
  }
  for (int t = threadIdx.x; t < N * CW; t += blockDim.x) {
    int c = t % CW, r = t / CW;
    if (c0 + c >= NC) continue;
    size_t o = inst + (size_t)r * NC + c0 + c;
    if constexpr (MODE == AX_FWD_ACC) {
      int col = c0 + c, p2 = col / HC, k3 = col % HC;
      int k1 = centred<N>(freq_of_pos<N>(r)), k2 = centred<N>(freq_of_pos<N>(p2));
      cpx<T> v = cscale(S[t], ((const T*)a.table)[k1 * k1 + k2 * k2 + k3 * k3]);
      dst[o] = a.first ? v : dst[o] + v;
    } else {
      dst[o] = S[t];
    }
  }
}

// out = L+ - uu M - ww g  (FP64), one CTA per (i1-plane, instance);
// zero-mode removal / conservation projection are done separately.
template <typename T, int N>
__global__ void __launch_bounds__(256) k_combine(const double* __restrict__ params, const double* __restrict__ g,
                                                 const T* __restrict__ Lp, const T* __restrict__ uu,
                                                 const T* __restrict__ ww, double* __restrict__ out, double h,
                                                 double log_inv_eps) {
  __shared__ double em[3 * N];
  __shared__ double thr;
  const int b = blockIdx.y, i1 = blockIdx.x;
  const InstanceParams q = load_params(params, b);
  fill_maxwellian_tables<N>(em, &thr, q, h, log_inv_eps);
  const double m1 = em[i1];
  const size_t base = ((size_t)b * N + i1) * N * N;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    int i2 = t / N, i3 = t % N;
    double M = m1 * em[N + i2] * em[2 * N + i3];
    size_t o = base + t;
    out[o] = (double)Lp[o] - (double)uu[o] * M - (double)ww[o] * g[o];
  }
}

}  // namespace lbo
