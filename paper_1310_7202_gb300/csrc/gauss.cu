// Step 1 of Algorithm 1: the Gaussian test matrix G (n x l, column-major).
//
// Random words: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11). Counter = (index lo32, index hi32, stream id, 0), key = (seed
// lo32, seed hi32). Element e = j*n + i of G takes word-pair (x0,x1) of counter e/4 for
// e%4 in {0,1} and (x2,x3) for e%4 in {2,3}.
//
// Normal deviates: Box-Muller, with the logarithm (atanh series after an exact binary
// split) and sine/cosine (Taylor series after an exact octant split) evaluated with
// explicitly rounded IEEE operations (__dadd_rn, __dmul_rn, ...) so that no FMA contraction
// changes the result: any implementation doing the same operations gets the same bits.
// Two variants: FP64 operations (FP64 path) and FP32 operations (FP32 and BF16 paths; one
// FP64 transform per pair would cost ~90 FP64 instructions, which GB300 runs at a small
// fraction of its FP32 rate).
#include "common.cuh"
#include "batched.cuh"

namespace rlu {

static constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
static constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
static constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
static constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Series coefficients, filled on the host by the recurrences stated at each field.
struct SeriesCoefs {
  double ln64[12];    // 1/(2n+1)
  double sin64[10];   // a_0 = 1, a_n = a_{n-1}/((2n)(2n+1)), alternating sign
  double cos64[10];   // b_0 = 1, b_n = b_{n-1}/((2n-1)(2n)), alternating sign
  float ln32[6];
  float sin32[7];
  float cos32[7];
};

static SeriesCoefs make_coefs() {
  SeriesCoefs c;
  for (int n = 0; n < 12; ++n) c.ln64[n] = 1.0 / (double)(2 * n + 1);
  double a = 1.0, b = 1.0;
  c.sin64[0] = 1.0;
  c.cos64[0] = 1.0;
  for (int n = 1; n < 10; ++n) {
    a = a / (double)((2 * n) * (2 * n + 1));
    b = b / (double)((2 * n - 1) * (2 * n));
    c.sin64[n] = (n & 1) ? -a : a;
    c.cos64[n] = (n & 1) ? -b : b;
  }
  for (int n = 0; n < 6; ++n) c.ln32[n] = 1.0f / (float)(2 * n + 1);
  float af = 1.0f, bf = 1.0f;
  c.sin32[0] = 1.0f;
  c.cos32[0] = 1.0f;
  for (int n = 1; n < 7; ++n) {
    af = af / (float)((2 * n) * (2 * n + 1));
    bf = bf / (float)((2 * n - 1) * (2 * n));
    c.sin32[n] = (n & 1) ? -af : af;
    c.cos32[n] = (n & 1) ? -bf : bf;
  }
  return c;
}

// ---- FP64 transform ------------------------------------------------------------------
__device__ __forceinline__ double ln_series64(double u, const SeriesCoefs& C) {
  const double kLn2 = 0x1.62e42fefa39efp-1, kSqrt2 = 0x1.6a09e667f3bcdp+0;
  int ex;
  const double mant = frexp(u, &ex);  // exact: u = mant * 2^ex, mant in [0.5, 1)
  double f = __dmul_rn(mant, 2.0);
  double e = (double)(ex - 1);
  if (f > kSqrt2) {
    f = mant;
    e = __dadd_rn(e, 1.0);
  }
  const double s = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
  const double z = __dmul_rn(s, s);
  double p = C.ln64[11];
#pragma unroll
  for (int n = 10; n >= 0; --n) p = __dadd_rn(__dmul_rn(p, z), C.ln64[n]);
  const double lnf = __dmul_rn(__dmul_rn(s, p), 2.0);
  return __dadd_rn(__dmul_rn(e, kLn2), lnf);
}

__device__ __forceinline__ void sincos_series64(uint32_t x, const SeriesCoefs& C, double& sn,
                                                double& cs) {
  const double kPi4 = 0x1.921fb54442d18p-1;
  const uint32_t q = x >> 29;
  double wi = (double)(x & ((1u << 29) - 1u));
  if (q & 1u) wi = __dsub_rn((double)(1u << 29), wi);
  const double phi = __dmul_rn(kPi4, __dmul_rn(wi, 0x1p-29));
  const double z = __dmul_rn(phi, phi);
  double sp = C.sin64[9], cp = C.cos64[9];
#pragma unroll
  for (int n = 8; n >= 0; --n) {
    sp = __dadd_rn(__dmul_rn(sp, z), C.sin64[n]);
    cp = __dadd_rn(__dmul_rn(cp, z), C.cos64[n]);
  }
  const double s = __dmul_rn(phi, sp), c = cp;
  switch (q) {
    case 0: sn = s; cs = c; break;
    case 1: sn = c; cs = s; break;
    case 2: sn = c; cs = -s; break;
    case 3: sn = s; cs = -c; break;
    case 4: sn = -s; cs = -c; break;
    case 5: sn = -c; cs = -s; break;
    case 6: sn = -c; cs = s; break;
    default: sn = -s; cs = c; break;
  }
}

__device__ __forceinline__ void box_muller64(uint32_t xa, uint32_t xb, const SeriesCoefs& C,
                                             double& z0, double& z1) {
  const double u = __dmul_rn(__dadd_rn((double)xa, 1.0), 0x1p-32);
  const double r = __dsqrt_rn(__dmul_rn(ln_series64(u, C), -2.0));
  double sn, cs;
  sincos_series64(xb, C, sn, cs);
  z0 = __dmul_rn(r, cs);
  z1 = __dmul_rn(r, sn);
}

// ---- FP32 transform ------------------------------------------------------------------
__device__ __forceinline__ void box_muller32(uint32_t xa, uint32_t xb, const SeriesCoefs& C,
                                             float& z0, float& z1) {
  const float kLn2 = 0x1.62e430p-1f, kSqrt2 = 0x1.6a09e6p+0f, kPi4 = 0x1.921fb6p-1f;
  const float u = __fmul_rn(__fadd_rn((float)(xa >> 8), 1.0f), 0x1p-24f);
  int ex;
  const float mant = frexpf(u, &ex);
  float f = __fmul_rn(mant, 2.0f);
  float e = (float)(ex - 1);
  if (f > kSqrt2) {
    f = mant;
    e = __fadd_rn(e, 1.0f);
  }
  const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
  const float z = __fmul_rn(s, s);
  float p = C.ln32[5];
#pragma unroll
  for (int n = 4; n >= 0; --n) p = __fadd_rn(__fmul_rn(p, z), C.ln32[n]);
  const float lnu = __fadd_rn(__fmul_rn(e, kLn2), __fmul_rn(__fmul_rn(s, p), 2.0f));
  const float r = __fsqrt_rn(__fmul_rn(lnu, -2.0f));

  const uint32_t q = xb >> 29;
  float wi = (float)((xb >> 5) & ((1u << 24) - 1u));
  if (q & 1u) wi = __fsub_rn((float)(1u << 24), wi);
  const float phi = __fmul_rn(kPi4, __fmul_rn(wi, 0x1p-24f));
  const float zz = __fmul_rn(phi, phi);
  float sp = C.sin32[6], cp = C.cos32[6];
#pragma unroll
  for (int n = 5; n >= 0; --n) {
    sp = __fadd_rn(__fmul_rn(sp, zz), C.sin32[n]);
    cp = __fadd_rn(__fmul_rn(cp, zz), C.cos32[n]);
  }
  const float sv = __fmul_rn(phi, sp), cv = cp;
  float sn, cs;
  switch (q) {
    case 0: sn = sv; cs = cv; break;
    case 1: sn = cv; cs = sv; break;
    case 2: sn = cv; cs = -sv; break;
    case 3: sn = sv; cs = -cv; break;
    case 4: sn = -sv; cs = -cv; break;
    case 5: sn = -cv; cs = -sv; break;
    case 6: sn = -cv; cs = sv; break;
    default: sn = -sv; cs = cv; break;
  }
  z0 = __fmul_rn(r, cs);
  z1 = __fmul_rn(r, sn);
}

// ---- kernels --------------------------------------------------------------------------
__global__ void k_philox_u32(uint64_t seed, uint32_t stream_id, uint64_t first,
                             int64_t n_counters, uint32_t* __restrict__ out) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_counters;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t idx = first + (uint64_t)c;
    const uint4 w = philox10(make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), stream_id, 0u),
                             k0, k1);
    reinterpret_cast<uint4*>(out)[c] = w;
  }
}

template <typename OutT>
__device__ __forceinline__ void store_g(OutT* G, int64_t ldg, int64_t n, int64_t e, float v);

template <>
__device__ __forceinline__ void store_g<float>(float* G, int64_t ldg, int64_t n, int64_t e,
                                               float v) {
  G[(e / n) * ldg + (e % n)] = v;
}
template <>
__device__ __forceinline__ void store_g<__nv_bfloat16>(__nv_bfloat16* G, int64_t ldg,
                                                       int64_t n, int64_t e, float v) {
  G[(e / n) * ldg + (e % n)] = __float2bfloat16_rn(v);
}

__global__ void k_gauss64(uint64_t seed, uint32_t stream_id, int64_t n, int64_t total,
                          double* __restrict__ G, int64_t ldg, SeriesCoefs C) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int64_t nc = (total + 3) / 4;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox10(make_uint4((uint32_t)c, (uint32_t)((uint64_t)c >> 32), stream_id,
                                        0u), k0, k1);
    double z[4];
    box_muller64(w.x, w.y, C, z[0], z[1]);
    box_muller64(w.z, w.w, C, z[2], z[3]);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t e = 4 * c + t;
      if (e < total) G[(e / n) * ldg + (e % n)] = z[t];
    }
  }
}

template <typename OutT>
__global__ void k_gauss32(uint64_t seed, uint32_t stream_id, int64_t n, int64_t total,
                          OutT* __restrict__ G, int64_t ldg, SeriesCoefs C) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int64_t nc = (total + 3) / 4;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox10(make_uint4((uint32_t)c, (uint32_t)((uint64_t)c >> 32), stream_id,
                                        0u), k0, k1);
    float z[4];
    box_muller32(w.x, w.y, C, z[0], z[1]);
    box_muller32(w.z, w.w, C, z[2], z[3]);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t e = 4 * c + t;
      if (e < total) store_g<OutT>(G, ldg, n, e, z[t]);
    }
  }
}

// Batched FP32 G: problem blockIdx.y of the table, its own seed and sizes.
__global__ void k_gauss32_batched(const GaussJob* __restrict__ jobs, SeriesCoefs C) {
  const GaussJob j = jobs[blockIdx.y];
  const uint32_t k0 = (uint32_t)j.seed, k1 = (uint32_t)(j.seed >> 32);
  const int64_t total = j.n * j.l, nc = (total + 3) / 4;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox10(make_uint4((uint32_t)c, (uint32_t)((uint64_t)c >> 32), 0u, 0u), k0,
                             k1);
    float z[4];
    box_muller32(w.x, w.y, C, z[0], z[1]);
    box_muller32(w.z, w.w, C, z[2], z[3]);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t e = 4 * c + t;
      if (e < total) j.G[(e / j.n) * j.ldg + (e % j.n)] = z[t];
    }
  }
}

int32_t launch_gaussian_batched(const GaussJob* jobs_dev, int count, cudaStream_t s) {
  if (count <= 0) return RLU_OK;
  if (count > 65535) return RLU_EINVAL;
  static const SeriesCoefs C = make_coefs();
  k_gauss32_batched<<<dim3(8, (unsigned)count), 256, 0, s>>>(jobs_dev, C);
  return last_launch_status();
}

static int grid_for(int64_t work, int threads) {
  const int64_t want = ceil_div(work, threads);
  const int64_t cap = (int64_t)sm_count() * 16;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

int32_t launch_gaussian(uint64_t seed, uint32_t stream_id, int64_t n, int64_t l, int32_t dtype,
                        void* G, int64_t ldg, cudaStream_t s) {
  const int64_t total = n * l;
  if (total == 0) return RLU_OK;
  static const SeriesCoefs C = make_coefs();
  const int threads = 256;
  const int grid = grid_for(ceil_div(total, 4), threads);
  if (dtype == RLU_F64) {
    k_gauss64<<<grid, threads, 0, s>>>(seed, stream_id, n, total, (double*)G, ldg, C);
  } else if (dtype == RLU_F32) {
    k_gauss32<float><<<grid, threads, 0, s>>>(seed, stream_id, n, total, (float*)G, ldg, C);
  } else if (dtype == RLU_BF16) {
    k_gauss32<__nv_bfloat16><<<grid, threads, 0, s>>>(seed, stream_id, n, total,
                                                      (__nv_bfloat16*)G, ldg, C);
  } else {
    return RLU_EUNSUPPORTED;
  }
  return last_launch_status();
}

}  // namespace rlu

extern "C" int32_t rlu_philox_u32(uint64_t seed, uint32_t stream_id, uint64_t first_counter,
                                  int64_t n_counters, uint32_t* out, void* stream) {
  if (out == nullptr || n_counters < 0) return RLU_EINVAL;
  if (((uintptr_t)out & 15u) != 0) return RLU_EINVAL;
  if (n_counters == 0) return RLU_OK;
  const int threads = 256;
  const int64_t want = rlu::ceil_div(n_counters, threads);
  const int64_t cap = (int64_t)rlu::sm_count() * 16;
  const int grid = (int)(want > cap ? cap : want);
  rlu::k_philox_u32<<<grid, threads, 0, (cudaStream_t)stream>>>(seed, stream_id, first_counter,
                                                                n_counters, out);
  return rlu::last_launch_status();
}

extern "C" int32_t rlu_gaussian(uint64_t seed, uint32_t stream_id, int64_t n, int64_t l,
                                int32_t dtype, void* G, int64_t ldg, void* stream) {
  if (G == nullptr || n < 0 || l < 0 || ldg < n || ldg < 1) return RLU_EINVAL;
  return rlu::launch_gaussian(seed, stream_id, n, l, dtype, G, ldg, (cudaStream_t)stream);
}
