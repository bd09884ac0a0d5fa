// Algorithm 4 of "Randomized LU Decomposition" (Section 4.1, fast randomized LU) on the GPU,
// in FP32 complex arithmetic (A real FP32; L and U complex):
//   1-2  Y = A R, R = D F S (Section 2, SRFT): k_srft_phase forms d_c = exp(2 pi i theta_c);
//        k_srft_rows multiplies a row of A by d, runs a mixed-radix (4, 2, 3, 5) Stockham FFT
//        in shared memory and keeps the l frequencies s_j, scaled by n^{-1/2}.
//   3    P Y = L_y U_y, partial pivoting on |Re| + |Im|: k_clu_coop, one cooperative launch
//        whose CTAs hold their rows in shared memory and meet at a grid barrier per step.
//   4-6  ID and B = L_y^+ P X A(J,:): with [L_1; L_2] the unit lower factor of step 3,
//        P X = [L_1; L_2] L_1^{-1}, J = P[:l], so B = M^{-1} V L_1^{-1} A(J,:) with
//        V = L_y^H [L_1; L_2] (k x l; its first k columns are M = L_y^H L_y). V is one real
//        product over the stacked real and imaginary planes (k_frlu_planes, FP32 products,
//        FP64 split reduction); W = V L_1^{-1} by k_frlu_wsolve (four warps per row); C = W A(J,:)
//        is one real product of the stacked planes of W with the gathered rows A(J,:); the
//        Hermitian system M B = C is solved through its real form [[Re M, -Im M], [Im M, Re M]]
//        by the LDL^T factorization and blocked substitution of Algorithm 1's step 5.
//   7    B Q = L_b U_b: the column-pivoted LU of B is the row-pivoted LU of B^T in the Crout
//        form (unit diagonal on the factor of B^T that becomes L_b): k_clu_coop again.
//   8-9  L = L_y L_b (one real product on the planes), U = U_b.
// Complex values are float2 (x = real part, y = imaginary part).
#include <algorithm>
#include <climits>
#include <cmath>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "panel_lu.cuh"
#include "small.cuh"
#include "umma.cuh"
#include "../../include/rlu_fast.h"

namespace rlu {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfms(float2 acc, float2 a, float2 b) {  // acc - a b
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// 1 / p without overflow or underflow of |p|^2 for moderate magnitudes: scale by max(|Re|, |Im|)
__device__ __forceinline__ float2 crecip(float2 p) {
  const float s = fmaxf(fabsf(p.x), fabsf(p.y));
  const float qx = p.x / s, qy = p.y / s;
  const float den = (qx * qx + qy * qy) * s;
  return make_float2(qx / den, -qy / den);
}

// ---------------------------------------------------------------------------------------
// Steps 1-2: the SRFT product Y = A D F S.
// ---------------------------------------------------------------------------------------

static constexpr int FFT_T = 512;    // threads per row transform
static constexpr int FFT_MAXV = 32;   // values per thread: n <= FFT_T * FFT_MAXV = 16384
                                      // (kernels for n <= 4096 and 8192 hold 8 and 16)
static constexpr int FFT_MAXST = 16;  // radix stages

struct FftPlan {
  int nst;
  int radix[FFT_MAXST];
};

// radices 4, 2, 3, 5 (all 4s first); false if n has another prime factor
static bool fft_plan(int n, FftPlan& p) {
  p.nst = 0;
  if (n < 1) return false;
  while (n % 4 == 0 && p.nst < FFT_MAXST) { p.radix[p.nst++] = 4; n /= 4; }
  for (int r : {2, 3, 5})
    while (n % r == 0 && p.nst < FFT_MAXST) { p.radix[p.nst++] = r; n /= r; }
  return n == 1;
}

// d_c = exp(2 pi i theta_c)
__global__ void k_srft_phase(const float* __restrict__ theta, int n, float2* __restrict__ d) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  float sn, cs;
  sincospif(2.f * theta[c], &sn, &cs);
  d[c] = make_float2(cs, sn);
}

// In-place P-point DFT of v (forward sign: X_q = sum_r v_r exp(-2 pi i q r / P)).
template <int P>
__device__ __forceinline__ void dft_small(float2 (&v)[P]);
template <>
__device__ __forceinline__ void dft_small<2>(float2 (&v)[2]) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void dft_small<4>(float2 (&v)[4]) {
  const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  const float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  v[1] = make_float2(d02.x + d13.y, d02.y - d13.x);  // d02 - i d13
  v[3] = make_float2(d02.x - d13.y, d02.y + d13.x);  // d02 + i d13
}
template <>
__device__ __forceinline__ void dft_small<3>(float2 (&v)[3]) {
  const float h = 0.86602540378443865f;  // sin(2 pi / 3)
  const float2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
  const float2 a = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  v[0] = cadd(v[0], t1);
  v[1] = make_float2(a.x + h * t2.y, a.y - h * t2.x);  // a - i h t2
  v[2] = make_float2(a.x - h * t2.y, a.y + h * t2.x);  // a + i h t2
}
template <>
__device__ __forceinline__ void dft_small<5>(float2 (&v)[5]) {
  // cos and sin of 2 pi q / 5 for q = 0..4
  const float c[5] = {1.f, 0.30901699437494742f, -0.80901699437494742f, -0.80901699437494742f,
                      0.30901699437494742f};
  const float s[5] = {0.f, 0.95105651629515357f, 0.58778525229247313f, -0.58778525229247313f,
                      -0.95105651629515357f};
  float2 x[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    float2 acc = v[0];
#pragma unroll
    for (int r = 1; r < 5; ++r) {
      const int e = (q * r) % 5;  // exp(-2 pi i e / 5) = c[e] - i s[e]
      acc.x += v[r].x * c[e] + v[r].y * s[e];
      acc.y += v[r].y * c[e] - v[r].x * s[e];
    }
    x[q] = acc;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) v[q] = x[q];
}

// One Stockham stage of radix P over buf (n values, natural order in and out after the
// last stage): butterfly j reads j + r n/P, twiddles by exp(-2 pi i (j mod Ns) r / (Ns P)),
// and writes (j / Ns) Ns P + (j mod Ns) + r Ns. All reads precede all writes (registers).
// The twiddle powers w^r come from repeated products: a few float ulps for r <= 4.
template <int P, int MAXV>
__device__ __forceinline__ void fft_stage(float2* buf, int n, int Ns) {
  constexpr int Q = (MAXV + P - 1) / P;
  const int nb = n / P;
  float2 v[Q][P];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = threadIdx.x + q * FFT_T;
    if (j < nb) {
#pragma unroll
      for (int r = 0; r < P; ++r) v[q][r] = buf[j + r * nb];
    }
  }
  __syncthreads();
  const float inv = 1.f / (float)(Ns * P);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = threadIdx.x + q * FFT_T;
    if (j < nb) {
      const int k = j % Ns;
      // twiddles w^r, w = exp(-2 pi i k / (Ns P)): one sincospif, powers by products
      float sn, cs;
      sincospif(-(float)(2 * k) * inv, &sn, &cs);
      const float2 w = make_float2(cs, sn);
      float2 wr = w;
#pragma unroll
      for (int r = 1; r < P; ++r) {
        v[q][r] = cmul(v[q][r], wr);
        if (r + 1 < P) wr = cmul(wr, w);
      }
      dft_small<P>(v[q]);
      const int d = (j / Ns) * Ns * P + k;
#pragma unroll
      for (int r = 0; r < P; ++r) buf[d + r * Ns] = v[q][r];
    }
  }
  __syncthreads();
}

// Row blockIdx.x of Y (row-major, ld ldy): Y[i][j] = scale * FFT(A[i, :] * d)[s_j].
// An index s_j outside [0, n) sets *status = RLU_EINVAL and yields 0.
template <int MAXV>
__global__ void __launch_bounds__(FFT_T) k_srft_rows(const float* __restrict__ A, int64_t lda,
                                                     int n, const float2* __restrict__ d,
                                                     const int32_t* __restrict__ sel, int l,
                                                     float scale, FftPlan plan,
                                                     float2* __restrict__ Y, int64_t ldy,
                                                     int32_t* __restrict__ status) {
  extern __shared__ __align__(16) float2 fbuf[];
  const int64_t row = blockIdx.x;
  const float* a = A + row * lda;
  {  // all of a thread's loads in flight before its stores
    float x[MAXV];
    float2 dc[MAXV];
#pragma unroll
    for (int q = 0; q < MAXV; ++q) {
      const int c = threadIdx.x + q * FFT_T;
      if (c < n) {
        x[q] = a[c];
        dc[q] = d[c];
      }
    }
#pragma unroll
    for (int q = 0; q < MAXV; ++q) {
      const int c = threadIdx.x + q * FFT_T;
      if (c < n) fbuf[c] = make_float2(x[q] * dc[q].x, x[q] * dc[q].y);
    }
  }
  __syncthreads();
  // the plan lists its radices grouped (4s, 2s, 3s, 5s): one loop per radix keeps each
  // stage's registers separate
  int Ns = 1, st = 0;
  for (; st < plan.nst && plan.radix[st] == 4; ++st, Ns *= 4) fft_stage<4, MAXV>(fbuf, n, Ns);
  for (; st < plan.nst && plan.radix[st] == 2; ++st, Ns *= 2) fft_stage<2, MAXV>(fbuf, n, Ns);
  for (; st < plan.nst && plan.radix[st] == 3; ++st, Ns *= 3) fft_stage<3, MAXV>(fbuf, n, Ns);
  for (; st < plan.nst && plan.radix[st] == 5; ++st, Ns *= 5) fft_stage<5, MAXV>(fbuf, n, Ns);
  for (int j = threadIdx.x; j < l; j += FFT_T) {
    const int sj = sel[j];
    float2 v = make_float2(0.f, 0.f);
    if (sj >= 0 && sj < n) {
      v = fbuf[sj];
      v.x *= scale;
      v.y *= scale;
    } else if (status) {
      *status = RLU_EINVAL;
    }
    Y[row * ldy + j] = v;
  }
}

// ---------------------------------------------------------------------------------------
// Steps 3 and 7: complex LU with partial pivoting, all min(rows, cols) steps, as one
// cooperative launch. CTA b holds rows [b R, b R + R) of the current order in shared memory
// (row-major, cols entries each). For step j:
//   * every CTA offers its best candidate of column j (first maximum of |Re| + |Im| at
//     positions >= j) by an atomicMax on a packed key (magnitude bits above the inverted
//     position, so that equal magnitudes go to the smaller position) and publishes the whole
//     candidate row; the owner of position j publishes row j;
//   * grid barrier (bounded wait: RLU_ETIMEOUT after 2 s);
//   * every CTA reads the key (the winner's CTA follows from its position), reads the pivot
//     row, performs the physical swap of rows j and r on the rows it owns, and updates its
//     rows below j: Doolittle (unit diagonal on L: multipliers divided by the pivot) for Y,
//     or Crout (unit diagonal on the pivot row: the row is divided by the pivot) for B^T.
// Look-ahead: the update first completes column j + 1, the candidate row of step j + 1 and
// the row at position j + 1, which are published before the rest of the update, so that
// the rest overlaps the barrier of step j + 1. Published rows are double-buffered by step
// parity (a CTA writes the buffer of step j + 2 only after the barrier of step j + 1, which
// every CTA passes after its reads of step j); keys rotate over three slots, slot (j + 2) % 3
// being cleared by CTA 0 after the barrier of step j. A zero pivot skips the swap and the
// update and is reported (LAPACK getf2).
// ---------------------------------------------------------------------------------------

static constexpr int CLU_T = 512;
static constexpr int CLU_TX = 32, CLU_TY = CLU_T / CLU_TX;
#ifndef RLU_CLU_MIN_ROWS
#define RLU_CLU_MIN_ROWS 8  // fewest rows per CTA (more rows: fewer CTAs meet at each step)
#endif

struct CluArgs {
  float2* Y;          // rows x cols, row-major, ld ldy; factored in place (position order)
  int64_t ldy;
  int rows, cols;
  int rloc;           // rows per CTA
  int32_t* perm;      // gather form: position i holds original row perm[i]
  float2* pub_rows;   // [2][G + 1][cols]
  int* pub_idx;       // [2][G + 1]
  unsigned long long* key;  // 3 slots, 128 bytes apart (own cache lines), zero before the launch
  unsigned* bar;      // zero before the launch
  int32_t* status;
  int32_t* first_zero;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t clu_now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// Arrival at the grid barrier: every thread's prior writes, then one increment.
__device__ __forceinline__ void clu_arrive(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
  }
}
// Wait until the counter reaches target; false (and RLU_ETIMEOUT in *status) when it does
// not within 2 s.
__device__ __forceinline__ bool clu_wait(unsigned* bar, unsigned target, int32_t* status,
                                         int* s_ok) {
  if (threadIdx.x == 0) {
    bool ok = true;
    if (ld_acquire_u32(bar) < target) {
      const uint64_t t0 = clu_now_ns();
      while (ld_acquire_u32(bar) < target) {
        if (clu_now_ns() - t0 > 2000000000ull) {
          ok = false;
          break;
        }
      }
    }
    __threadfence();
    if (!ok && status) atomicExch(status, RLU_ETIMEOUT);
    *s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Packed candidate: |Re| + |Im| (non-negative, so its bits order like the values) above
// the inverted position; 0 means no candidate.
__device__ __forceinline__ unsigned long long clu_pack(float mag, int pos) {
  return ((unsigned long long)__float_as_uint(mag) << 32) | (unsigned)(0xFFFFFFFFu - (unsigned)pos);
}

template <bool CROUT>
__device__ __forceinline__ void clu_candidate(const float2* tile, int cols, int nloc, int base,
                                              int col, int* s_cpos, unsigned long long* key) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    float mag = -1.f;
    int pos = INT_MAX;
    for (int r = lane; r < nloc; r += 32) {
      const int p = base + r;
      if (p < col) continue;
      const float2 v = tile[(size_t)r * cols + col];
      const float mg = fabsf(v.x) + fabsf(v.y);
      if (cand_better(mg, p, mag, pos)) {
        mag = mg;
        pos = p;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float om = __shfl_xor_sync(0xffffffffu, mag, off);
      const int op = __shfl_xor_sync(0xffffffffu, pos, off);
      if (cand_better(om, op, mag, pos)) {
        mag = om;
        pos = op;
      }
    }
    if (lane == 0) {
      *s_cpos = pos;
      if (pos != INT_MAX) atomicMax(key, clu_pack(mag, pos));
    }
  }
}

// Publish the candidate row (if any) and the row at position col (if owned) for step col.
__device__ __forceinline__ void clu_publish(const float2* tile, const int* idx, int cols,
                                            int nloc, int base, int col, int cpos, int b, int G,
                                            float2* prow, int* pidx) {
  if (cpos != INT_MAX) {
    const float2* src = tile + (size_t)(cpos - base) * cols;
    for (int c = threadIdx.x; c < cols; c += CLU_T) prow[(size_t)b * cols + c] = src[c];
    if (threadIdx.x == 0) pidx[b] = idx[cpos - base];
  }
  if (col >= base && col < base + nloc) {
    const float2* src = tile + (size_t)(col - base) * cols;
    for (int c = threadIdx.x; c < cols; c += CLU_T) prow[(size_t)G * cols + c] = src[c];
    if (threadIdx.x == 0) pidx[G] = idx[col - base];
  }
}

template <bool CROUT>
__global__ void __launch_bounds__(CLU_T, 1) k_clu_coop(CluArgs a) {
  extern __shared__ __align__(16) unsigned char clu_smem[];
  const int cols = a.cols;
  float2* tile = reinterpret_cast<float2*>(clu_smem);         // [rloc][cols]
  float2* piv = tile + (size_t)a.rloc * cols;                   // [cols]
  int* idx = reinterpret_cast<int*>(piv + cols);                // [rloc]
  __shared__ int s_ok, s_cpos, s_w, s_r;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int base = b * a.rloc;
  const int nloc = max(0, min(a.rloc, a.rows - base));
  const int steps = min(a.rows, cols);
  const int tx = tid % CLU_TX, ty = tid / CLU_TX;
  for (int e = tid; e < nloc * cols; e += CLU_T)
    tile[e] = a.Y[(int64_t)(base + e / cols) * a.ldy + e % cols];
  for (int r = tid; r < nloc; r += CLU_T) idx[r] = base + r;
  __syncthreads();
  // step 0's candidates
  clu_candidate<CROUT>(tile, cols, nloc, base, 0, &s_cpos, a.key);
  __syncthreads();
  clu_publish(tile, idx, cols, nloc, base, 0, s_cpos, b, G, a.pub_rows, a.pub_idx);
  clu_arrive(a.bar);
  for (int j = 0; j < steps; ++j) {
    const int par = j & 1;
    const float2* prow = a.pub_rows + (size_t)par * (G + 1) * cols;
    const int* pidx = a.pub_idx + (size_t)par * (G + 1);
    if (!clu_wait(a.bar, (unsigned)G * (unsigned)(j + 1), a.status, &s_ok)) return;
    if (tid == 0) {
      const unsigned long long kv = __ldcg(a.key + 16 * (j % 3));
      const float mag = __uint_as_float((unsigned)(kv >> 32));
      const int pos = (int)(0xFFFFFFFFu - (unsigned)(kv & 0xFFFFFFFFu));
      const bool valid = kv != 0ull && pos >= j && pos < a.rows;
      s_w = (valid && mag > 0.f) ? pos / a.rloc : -1;  // zero (or no finite) pivot: -1
      s_r = pos;
      if (b == 0) a.key[16 * ((j + 2) % 3)] = 0ull;             // the slot of step j + 2
    }
    __syncthreads();
    const int w = s_w, r = s_r;
    const bool last = j + 1 >= steps;
    const int parn = (j + 1) & 1;
    float2* prown = a.pub_rows + (size_t)parn * (G + 1) * cols;
    int* pidxn = a.pub_idx + (size_t)parn * (G + 1);
    if (w < 0) {  // nothing to eliminate: the next step's candidates as they stand
      if (b == 0 && tid == 0 && a.first_zero) atomicCAS(a.first_zero, -1, j);
      if (!last) {
        clu_candidate<CROUT>(tile, cols, nloc, base, j + 1, &s_cpos, a.key + 16 * ((j + 1) % 3));
        __syncthreads();
        clu_publish(tile, idx, cols, nloc, base, j + 1, s_cpos, b, G, prown, pidxn);
        clu_arrive(a.bar);
      }
      continue;
    }
    const float2* wsrc = prow + (size_t)w * cols;
    for (int c = tid; c < cols; c += CLU_T) piv[c] = __ldcg(wsrc + c);
    __syncthreads();
    const float2 pinv = crecip(piv[j]);
    if (CROUT) {
      for (int c = j + 1 + tid; c < cols; c += CLU_T) piv[c] = cmul(piv[c], pinv);
      __syncthreads();
    }
    // the swap of positions j and r, on the rows this CTA owns
    if (r != j && r >= base && r < base + nloc) {
      const float2* src = prow + (size_t)G * cols;
      for (int c = tid; c < cols; c += CLU_T) tile[(size_t)(r - base) * cols + c] = __ldcg(src + c);
      if (tid == 0) idx[r - base] = __ldcg(pidx + G);
    }
    if (j >= base && j < base + nloc) {
      for (int c = tid; c < cols; c += CLU_T) tile[(size_t)(j - base) * cols + c] = piv[c];
      if (tid == 0) idx[j - base] = __ldcg(pidx + w);
    }
    __syncthreads();
    // rows below position j: multipliers (Doolittle) and column j + 1
    const int r0 = max(j + 1 - base, 0);
    for (int rr = r0 + tid; rr < nloc; rr += CLU_T) {
      float2* trow = tile + (size_t)rr * cols;
      float2 lv = trow[j];
      if (!CROUT) {
        lv = cmul(lv, pinv);
        trow[j] = lv;
      }
      if (!last) trow[j + 1] = cfms(trow[j + 1], lv, piv[j + 1]);
    }
    __syncthreads();
    int ca = -1, cb = -1;  // local rows updated ahead of the others
    if (!last) {
      clu_candidate<CROUT>(tile, cols, nloc, base, j + 1, &s_cpos, a.key + 16 * ((j + 1) % 3));
      __syncthreads();
      const int cpos = s_cpos;
      ca = cpos != INT_MAX ? cpos - base : -1;
      cb = (j + 1 >= base && j + 1 < base + nloc) ? j + 1 - base : -1;
      if (cb == ca) cb = -1;
      // complete the two rows the next step publishes (warp 0: ca, warp 1: cb)
      const int wid = tid >> 5, lane = tid & 31;
      const int rr = wid == 0 ? ca : (wid == 1 ? cb : -1);
      if (rr >= 0) {
        float2* trow = tile + (size_t)rr * cols;
        const float2 lv = trow[j];
        for (int c = j + 2 + lane; c < cols; c += 32) trow[c] = cfms(trow[c], lv, piv[c]);
      }
      __syncthreads();
      clu_publish(tile, idx, cols, nloc, base, j + 1, cpos, b, G, prown, pidxn);
      clu_arrive(a.bar);
    }
    // the rest of the update overlaps the barrier of step j + 1
    const int c0 = last ? j + 1 : j + 2;
    for (int rr = r0 + ty; rr < nloc; rr += CLU_TY) {
      if (rr == ca || rr == cb) continue;
      float2* trow = tile + (size_t)rr * cols;
      const float2 lv = trow[j];
      for (int c = c0 + tx; c < cols; c += CLU_TX) trow[c] = cfms(trow[c], lv, piv[c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < nloc * cols; e += CLU_T)
    a.Y[(int64_t)(base + e / cols) * a.ldy + e % cols] = tile[e];
  for (int r = tid; r < nloc; r += CLU_T) a.perm[base + r] = idx[r];
}

static size_t clu_smem_bytes(int rloc, int cols) {
  return (size_t)rloc * cols * sizeof(float2) + (size_t)cols * sizeof(float2) +
         (size_t)rloc * sizeof(int);
}

// Workspace of the barrier, the keys and the published rows for up to G CTAs.
static constexpr int CLU_HDR = 512;  // barrier counter and three key slots, a line each
static size_t clu_pub_bytes(int G, int cols) {
  return CLU_HDR + 2 * (size_t)(G + 1) * cols * sizeof(float2) + 2 * (size_t)(G + 1) * sizeof(int);
}

// CTAs and rows per CTA for a rows x cols LU; false when the rows do not fit.
static bool clu_shape(int rows, int cols, int* G, int* rloc) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  if (rows < 1) return false;
  int g = (int)ceil_div(rows, RLU_CLU_MIN_ROWS);
  if (g > sm_count()) g = sm_count();
  if (g < 1) g = 1;
  const int r = (int)ceil_div(rows, g);
  if (clu_smem_bytes(r, cols) + 1024 > (size_t)optin) return false;
  *G = (int)ceil_div(rows, r);
  *rloc = r;
  return true;
}

static int32_t clu_coop(bool crout, float2* Y, int64_t ldy, int rows, int cols, int32_t* perm,
                        void* pub, int pub_G, int32_t* status, int32_t* first_zero,
                        cudaStream_t s) {
  int G = 0, rloc = 0;
  if (!clu_shape(rows, cols, &G, &rloc) || G > pub_G) return RLU_EUNSUPPORTED;
  char* p = static_cast<char*>(pub);
  CluArgs a{};
  a.Y = Y;
  a.ldy = ldy;
  a.rows = rows;
  a.cols = cols;
  a.rloc = rloc;
  a.perm = perm;
  a.bar = reinterpret_cast<unsigned*>(p);                      // header: barrier, 3 keys
  a.key = reinterpret_cast<unsigned long long*>(p + 128);
  p += CLU_HDR;
  a.pub_rows = reinterpret_cast<float2*>(p);
  p += 2 * (size_t)(G + 1) * cols * sizeof(float2);
  a.pub_idx = reinterpret_cast<int*>(p);
  a.status = status;
  a.first_zero = first_zero;
  const size_t smem = clu_smem_bytes(rloc, cols);
  const void* fn = crout ? reinterpret_cast<const void*>(&k_clu_coop<true>)
                         : reinterpret_cast<const void*>(&k_clu_coop<false>);
  RLU_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  RLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, CLU_T, smem));
  if (per_sm * sm_count() < G) return RLU_EUNSUPPORTED;
  RLU_CUDA_TRY(cudaMemsetAsync(a.bar, 0, CLU_HDR, s));
  void* args[] = {&a};
  RLU_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(CLU_T), args, smem, s));
  return last_launch_status();
}

// ---------------------------------------------------------------------------------------
// Steps 4-9: planes, products and small solves around the two LUs.
// ---------------------------------------------------------------------------------------

// S (2m x 2l, column-major, ld 2m) from the factored Y (unit lower factor L_f = [L_1; L_2],
// m x l): column j = [Re L_f[:, j]; Im L_f[:, j]], column l + j = [Im L_f[:, j]; -Re L_f[:, j]].
// Then V = S[:, :k]^T S = [Re V | Im V] with V = L_y^H L_f, and viewed with ld m, the first 2k
// columns of S are Re L_y[:, 0], Im L_y[:, 0], Re L_y[:, 1], ... (the operand of L = L_y L_b).
__global__ void k_frlu_planes(const float2* __restrict__ Y, int64_t ldy, int m, int l,
                              float* __restrict__ S) {
  __shared__ float2 t[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int yy = ty; yy < 32; yy += 8) {
    const int i = i0 + yy, j = j0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (i < m && j < l) {
      if (i > j) v = Y[(int64_t)i * ldy + j];
      else if (i == j) v = make_float2(1.f, 0.f);
    }
    t[yy][tx] = v;
  }
  __syncthreads();
  const int64_t ld2 = 2 * (int64_t)m;
  for (int yy = ty; yy < 32; yy += 8) {
    const int j = j0 + yy, i = i0 + tx;
    if (j < l && i < m) {
      const float2 v = t[tx][yy];
      float* c1 = S + (int64_t)j * ld2;
      float* c2 = S + (int64_t)(l + j) * ld2;
      c1[i] = v.x;
      c1[m + i] = v.y;
      c2[i] = v.y;
      c2[m + i] = -v.x;
    }
  }
}

// Real form [[Re M, -Im M], [Im M, Re M]] (2k x 2k, row-major) of the Hermitian Gram
// M = V[:, :k], taken from its lower triangle so that the real form is exactly symmetric.
__global__ void k_frlu_embed(const double* __restrict__ V, int64_t ldv, int k, int l,
                             double* __restrict__ Mre) {
  const int64_t k2 = 2 * (int64_t)k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k2 * k2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a2 = (int)(e / k2), b2 = (int)(e % k2);
    const int a = a2 % k, bb = b2 % k;
    double mr, mi;
    if (a >= bb) {
      mr = V[(int64_t)a * ldv + bb];
      mi = V[(int64_t)a * ldv + l + bb];
    } else {
      mr = V[(int64_t)bb * ldv + a];
      mi = -V[(int64_t)bb * ldv + l + a];
    }
    const bool ai = a2 >= k, bi = b2 >= k;
    Mre[e] = (ai == bi) ? mr : (bi ? -mi : mi);
  }
}

// W = V L_1^{-1} (k x l) for the unit lower L_1 (the leading l x l block of the factored Y):
// row a solves w L_1 = V[a, :] by 32-column blocks from the last. Each row is held by
// WS_PARTS warps: lane t of part q holds the entries c = lane + 32 s for the blocks
// s = q + WS_PARTS u (u < NS / WS_PARTS, l <= 32 NS). For block sb the CTA stages rows
// 32 sb .. 32 sb + 31 of L_1 (columns up to the block's end) in shared memory; the part that
// holds the block finalises its columns from the last down (w_b = v_b, then
// v_c -= w_b L_1[b][c] for c < b inside the block) and shares the 32 values w; then every
// part updates its blocks left of sb, v_c -= sum_b w_b L_1[b][c]. Writes the planes
// Wst[a] = Re w, Wst[k + a] = Im w (2k x l row-major, ld ldw).
static constexpr int WS_ROWS = 4;   // rows of W per CTA
static constexpr int WS_PARTS = 4;  // warps per row
static constexpr int WS_T = 32 * WS_ROWS * WS_PARTS;

template <int NS>
__global__ void __launch_bounds__(WS_T) k_frlu_wsolve(const double* __restrict__ V, int64_t ldv,
                                                      int k, int l, const float2* __restrict__ Y,
                                                      int64_t ldy, float* __restrict__ Wst,
                                                      int64_t ldw) {
  extern __shared__ __align__(16) float2 ws_rows[];  // [32][32 NS]
  __shared__ float2 wbuf[WS_ROWS][32];
  constexpr int LDS = 32 * NS;
  constexpr int NU = (NS + WS_PARTS - 1) / WS_PARTS;  // blocks per part
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = warp / WS_PARTS, q = warp % WS_PARTS;
  const int a = blockIdx.x * WS_ROWS + row;
  const bool active = a < k;
  float2 v[NU];
#pragma unroll
  for (int u = 0; u < NU; ++u) {
    const int c = lane + 32 * (q + WS_PARTS * u);
    v[u] = (active && c < l)
               ? make_float2((float)V[(int64_t)a * ldv + c], (float)V[(int64_t)a * ldv + l + c])
               : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int sb = NS - 1; sb >= 0; --sb) {
    if (32 * sb >= l) continue;  // the same for every thread
    const int ncol = min(32 * sb + 32, l);
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += WS_T) {  // 8 independent loads in flight
#pragma unroll
      for (int i0 = 0; i0 < 32; i0 += 8) {
        float2 t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int bi = 32 * sb + i0 + u;
          t[u] = bi < l ? Y[(int64_t)bi * ldy + c] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) ws_rows[(i0 + u) * LDS + c] = t[u];
      }
    }
    __syncthreads();
    // the part holding block sb solves it
    if (q == sb % WS_PARTS) {
      float2 x = v[sb / WS_PARTS];
      for (int li = 31; li >= 0; --li) {
        if (32 * sb + li >= l) continue;
        const float2 wb = make_float2(__shfl_sync(0xffffffffu, x.x, li),
                                      __shfl_sync(0xffffffffu, x.y, li));
        if (lane < li) x = cfms(x, wb, ws_rows[li * LDS + 32 * sb + lane]);
      }
      v[sb / WS_PARTS] = x;
      wbuf[row][lane] = x;
    }
    __syncthreads();
    if (sb > 0) {
      for (int bb = 0; bb < 32; ++bb) {
        if (32 * sb + bb >= l) break;
        const float2 wb = wbuf[row][bb];
        const float2* Lrow = ws_rows + bb * LDS + lane;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int sblk = q + WS_PARTS * u;
          if (sblk < sb) v[u] = cfms(v[u], wb, Lrow[32 * sblk]);
        }
      }
    }
  }
  if (!active) return;
#pragma unroll
  for (int u = 0; u < NU; ++u) {
    const int c = lane + 32 * (q + WS_PARTS * u);
    if (c < l) {
      Wst[(int64_t)a * ldw + c] = v[u].x;
      Wst[(int64_t)(k + a) * ldw + c] = v[u].y;
    }
  }
}

template <int NS>
static int32_t wsolve_launch(const double* V, int64_t ldv, int k, int l, const float2* Y,
                             int64_t ldy, float* Wst, int64_t ldw, cudaStream_t s) {
  const size_t smem = 32 * 32 * NS * sizeof(float2);
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_frlu_wsolve<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  k_frlu_wsolve<NS><<<(unsigned)ceil_div(k, WS_ROWS), WS_T, smem, s>>>(V, ldv, k, l, Y, ldy, Wst,
                                                                       ldw);
  return last_launch_status();
}

// A(J,:) (l x n, row-major, ld ldaj): row i is row perm[i] of A.
__global__ void k_frlu_gather_aj(const float* __restrict__ A, int64_t lda, int n,
                                 const int32_t* __restrict__ perm, float* __restrict__ AJ,
                                 int64_t ldaj) {
  const int i = blockIdx.y;
  const int64_t src = perm[i];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
    AJ[(int64_t)i * ldaj + c] = A[src * lda + c];
}

// B^T (n x k complex, row-major, ld ldt) from the planes Bst = [Re B; Im B] (2k x n, ld ldb).
__global__ void k_frlu_pack_bt(const float* __restrict__ Bst, int64_t ldb, int k, int n,
                               float2* __restrict__ Bt, int64_t ldt) {
  __shared__ float2 t[32][33];
  const int c0 = blockIdx.x * 32, j0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int yy = ty; yy < 32; yy += 8) {
    const int j = j0 + yy, c = c0 + tx;
    t[yy][tx] = (j < k && c < n) ? make_float2(Bst[(int64_t)j * ldb + c], Bst[(int64_t)(k + j) * ldb + c])
                                 : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int c = c0 + yy, j = j0 + tx;
    if (c < n && j < k) Bt[(int64_t)c * ldt + j] = t[tx][yy];
  }
}

// U = U_b (k x n complex, row-major, ld ldu) from the Crout-factored B^T: U[j][c] = Bt[c][j]
// for c >= j (the factor of B^T that carries the pivots), 0 below the diagonal.
__global__ void k_frlu_unpack_u(const float2* __restrict__ Bt, int64_t ldt, int k, int n,
                                float2* __restrict__ U, int64_t ldu) {
  __shared__ float2 t[32][33];
  const int c0 = blockIdx.x * 32, j0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int yy = ty; yy < 32; yy += 8) {
    const int c = c0 + yy, j = j0 + tx;
    t[yy][tx] = (c < n && j < k) ? Bt[(int64_t)c * ldt + j] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int j = j0 + yy, c = c0 + tx;
    if (j < k && c < n) U[(int64_t)j * ldu + c] = (c >= j) ? t[tx][yy] : make_float2(0.f, 0.f);
  }
}

// Real form of L_b (unit lower, L_b[c][j] = Bt[j][c] for c > j) as the operand of
// L = L_y L_b on the planes: rows 2c and 2c + 1 multiply Re and Im of column c of L_y;
// columns j and k + j produce Re and Im of column j of L (2k x 2k, row-major).
__global__ void k_frlu_lb_embed(const float2* __restrict__ Bt, int64_t ldt, int k,
                                float* __restrict__ Lbe) {
  const int64_t kk = (int64_t)k * k;
  const int64_t k2 = 2 * (int64_t)k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kk;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / k), c = (int)(e % k);
    float2 v = make_float2(0.f, 0.f);
    if (c > j) v = Bt[(int64_t)j * ldt + c];
    else if (c == j) v = make_float2(1.f, 0.f);
    Lbe[(2 * c) * k2 + j] = v.x;
    Lbe[(2 * c + 1) * k2 + j] = -v.y;
    Lbe[(2 * c) * k2 + k + j] = v.y;
    Lbe[(2 * c + 1) * k2 + k + j] = v.x;
  }
}

// L (m x k complex, column-major, ld ldl) from [Re L | Im L] (m x 2k, column-major, ld m).
__global__ void k_frlu_pack_l(const float* __restrict__ Lo, int m, int k, float2* __restrict__ L,
                              int64_t ldl) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    L[(int64_t)j * ldl + i] = make_float2(Lo[(int64_t)j * m + i], Lo[(int64_t)(k + j) * m + i]);
}

// Row-major R x C complex (ld ldr) -> column-major (ld ldc), through a 32 x 32 shared tile.
__global__ void k_c_rm_to_cm(const float2* __restrict__ Yr, int64_t ldr, int R, int C,
                             float2* __restrict__ X, int64_t ldc) {
  __shared__ float2 t[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < C) t[i][threadIdx.x] = Yr[(int64_t)r * ldr + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j, r = r0 + threadIdx.x;
    if (r < R && c < C) X[(int64_t)c * ldc + r] = t[threadIdx.x][j];
  }
}

// The register LU's swap-free result back to the positional row-major layout of the rest of
// the pipeline: row p of Yr = row perm[p] of X (column-major, ld ldc).
__global__ void k_c_cm_to_rm_perm(const float2* __restrict__ X, int64_t ldc, int R, int C,
                                  const int32_t* __restrict__ perm, float2* __restrict__ Yr,
                                  int64_t ldr) {
  __shared__ float2 t[32][33];
  __shared__ int src[32];
  const int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  if (threadIdx.y == 0) src[threadIdx.x] = p0 + threadIdx.x < R ? perm[p0 + threadIdx.x] : 0;
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {  // column c0 + j, rows src[x]
    const int c = c0 + j, p = p0 + threadIdx.x;
    if (p < R && c < C) t[threadIdx.x][j] = X[(int64_t)c * ldc + src[threadIdx.x]];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int p = p0 + i, c = c0 + threadIdx.x;
    if (p < R && c < C) Yr[(int64_t)p * ldr + c] = t[i][threadIdx.x];
  }
}

// Exact TF32 parts (hi = x with its 13 low mantissa bits cleared, lo = x - hi) of the
// transpose of a row-major R x C matrix: hi / lo[c * ldo + r] from X[r * ldx + c].
__global__ void k_split_t(const float* __restrict__ X, int64_t ldx, int R, int C,
                          float* __restrict__ hi, float* __restrict__ lo, int64_t ldo) {
  __shared__ float t[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (r < R && c < C) ? X[(int64_t)r * ldx + c] : 0.f;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j, r = r0 + threadIdx.x;
    if (r < R && c < C) {
      const float v = t[threadIdx.x][j];
      const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
      hi[(int64_t)c * ldo + r] = h;
      lo[(int64_t)c * ldo + r] = v - h;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Workspace plan and the entry points.
// ---------------------------------------------------------------------------------------

struct FastPlan {
  int64_t ldn = 0;  // row length of the n-wide planes
  int kp = 0, split_v = 1, ns = 1;
  FftPlan fft{};
  size_t off_d = 0, off_Y = 0, off_pub = 0, off_S = 0, off_V = 0, off_part = 0, off_M = 0,
         off_LT = 0, off_LR = 0, off_W = 0, off_WT = 0, off_dinv = 0, off_Wst = 0, off_AJ = 0,
         off_C = 0, off_B = 0, off_Bt = 0, off_Lbe = 0, off_Lo = 0, total = 0;
  // the register LU's column-major copy of Y (then of B^T), position state, pivot rows
  size_t off_X = 0, off_posg = 0, off_psg = 0, off_u12 = 0;
  int64_t ldxy = 0, ldxb = 0, ldu12 = 0;
  // the three plane products on the tensor cores (TF32 splits of their second operands,
  // FP32 partial slices) when every leading dimension suits TMA
  bool tc = false;
  int split_vt = 1;
  size_t off_Sh = 0, off_Sl = 0, off_Wh = 0, off_Wl = 0, off_Lbh = 0, off_Lbl = 0, off_part2 = 0;
};

static size_t fp_carve(size_t& cur, size_t bytes) {
  const size_t at = cur;
  cur += (size_t)round_up((int64_t)bytes, 256);
  return at;
}

// RLU_OK, RLU_EINVAL (sizes) or RLU_EUNSUPPORTED (outside the kernels' limits).
static int32_t fast_plan(int64_t m, int64_t n, int k, int l, FastPlan& p) {
  if (m < 1 || n < 1 || k < 1 || k > l || l > m || l > n) return RLU_EINVAL;
  if (m > INT_MAX / 2 || n > INT_MAX / 2) return RLU_EUNSUPPORTED;
  if (n > (int64_t)FFT_T * FFT_MAXV || !fft_plan((int)n, p.fft)) return RLU_EUNSUPPORTED;
  if (l > 512 || !ldl_factor_supported(2 * k, true)) return RLU_EUNSUPPORTED;
  int G = 0, rloc = 0;
  if (!clu_shape((int)m, l, &G, &rloc) || !clu_shape((int)n, k, &G, &rloc)) return RLU_EUNSUPPORTED;
  p.ns = l <= 32 ? 1 : l <= 64 ? 2 : l <= 128 ? 4 : l <= 256 ? 8 : 16;
  p.ldn = round_up(n, 4);
  p.kp = (int)round_up(2 * (int64_t)k, 32);
  const int64_t tiles = ceil_div(k, gemm_tile_m(RLU_F32)) * ceil_div(2 * (int64_t)l, gemm_tile_n(RLU_F32));
  int64_t sp = ceil_div(2 * (int64_t)sm_count(), tiles);
  const int64_t kmax = (2 * m) / 64 > 1 ? (2 * m) / 64 : 1;
  sp = sp > kmax ? kmax : sp;
  p.split_v = (int)(sp < 2 ? 2 : sp);  // FP32 partials, FP64 reduction
  const int64_t k2 = 2 * (int64_t)k;
  size_t cur = 0;
  p.off_d = fp_carve(cur, (size_t)n * sizeof(float2));
  p.off_Y = fp_carve(cur, (size_t)m * l * sizeof(float2));
  p.off_pub = fp_carve(cur, clu_pub_bytes(sm_count(), l));
  p.off_S = fp_carve(cur, (size_t)(2 * m) * (2 * l) * sizeof(float));
  p.off_V = fp_carve(cur, (size_t)k * (2 * l) * sizeof(double));
  p.off_part = fp_carve(cur, gemm_partial_bytes<float>(k, 2 * (int64_t)l, p.split_v));
  p.off_M = fp_carve(cur, (size_t)k2 * k2 * sizeof(double));
  p.off_LT = fp_carve(cur, (size_t)p.kp * p.kp * sizeof(float));
  p.off_LR = fp_carve(cur, (size_t)p.kp * p.kp * sizeof(float));
  p.off_W = fp_carve(cur, (size_t)p.kp * 32 * sizeof(float));
  p.off_WT = fp_carve(cur, (size_t)p.kp * 32 * sizeof(float));
  p.off_dinv = fp_carve(cur, (size_t)k2 * sizeof(double));
  p.off_Wst = fp_carve(cur, (size_t)k2 * l * sizeof(float));
  p.off_AJ = fp_carve(cur, (size_t)l * p.ldn * sizeof(float));
  p.off_C = fp_carve(cur, (size_t)k2 * p.ldn * sizeof(float));
  p.off_B = fp_carve(cur, (size_t)k2 * p.ldn * sizeof(float));
  p.off_Bt = fp_carve(cur, (size_t)n * k * sizeof(float2));
  p.off_Lbe = fp_carve(cur, (size_t)k2 * k2 * sizeof(float));
  p.off_Lo = fp_carve(cur, (size_t)m * k2 * sizeof(float));
  p.ldxy = round_up(m, 4);
  p.ldxb = round_up(n, 4);
  p.ldu12 = round_up(l, 4);
  p.off_X = fp_carve(cur, (size_t)std::max(p.ldxy * l, p.ldxb * k) * sizeof(float2));
  p.off_posg = fp_carve(cur, (size_t)std::max(m, n) * sizeof(int32_t));
  p.off_psg = fp_carve(cur, (size_t)l * sizeof(int32_t));
  p.off_u12 = fp_carve(cur, (size_t)96 * p.ldu12 * sizeof(float2));
  p.tc = m % 4 == 0 && l % 4 == 0 && k % 2 == 0 && p.ldn % 4 == 0;
  if (p.tc) {
    p.split_vt = umma3_splits(k, 2 * m, 2 * (int64_t)l);
    const int64_t kc = round_up(ceil_div(2 * m, p.split_vt), 32);
    const int64_t sv = ceil_div(2 * m, kc);
    p.off_Sh = fp_carve(cur, (size_t)(2 * m) * (2 * l) * sizeof(float));
    p.off_Sl = fp_carve(cur, (size_t)(2 * m) * (2 * l) * sizeof(float));
    p.off_Wh = fp_carve(cur, (size_t)k2 * l * sizeof(float));
    p.off_Wl = fp_carve(cur, (size_t)k2 * l * sizeof(float));
    p.off_Lbh = fp_carve(cur, (size_t)k2 * k2 * sizeof(float));
    p.off_Lbl = fp_carve(cur, (size_t)k2 * k2 * sizeof(float));
    p.off_part2 = fp_carve(cur, std::max<size_t>((size_t)sv * k * (2 * l),
                                                 (size_t)2 * std::max(m, n) * k2) *
                                    sizeof(float));
  }
  p.total = cur;
  return RLU_OK;
}

// Steps 3 and 7: the pivoted LU (|Re| + |Im| pivots) of a tall complex matrix, row-major
// R x C (ld ldy), in place: on return row p holds the factors of position p and perm[p] the
// original row there. The cluster register LU (lu_reg.cu, complex FP32) factors a
// column-major copy, swap-free, and the result is gathered back; where it does not launch
// (shape), the cooperative kernel factors Y directly.
static int32_t clu_factor(const FastPlan& p, char* ws, bool crout, float2* Y, int64_t ldy, int R,
                          int C, int32_t* perm, void* pub, int32_t* status, int32_t* nonfinite,
                          int32_t* first_zero, cudaStream_t s) {
  const int64_t ldx = round_up(R, 4);
  float2* X = reinterpret_cast<float2*>(ws + p.off_X);
  const dim3 tb(32, 8), tg((unsigned)ceil_div(R, 32), (unsigned)ceil_div(C, 32));
  k_c_rm_to_cm<<<tg, tb, 0, s>>>(Y, ldy, R, C, X, ldx);
  RLU_TRY(last_launch_status());
  LuArgs a{};
  a.X = X;
  a.ldx = ldx;
  a.R = R;
  a.C = C;
  a.perm = perm;
  a.zero_step = first_zero;
  a.nonfinite = nonfinite;
  a.status = status;
  a.posg = reinterpret_cast<int32_t*>(ws + p.off_posg);
  a.psg = reinterpret_cast<int32_t*>(ws + p.off_psg);
  a.u12 = ws + p.off_u12;
  a.ldu = p.ldu12;
  bool launched = false;
  RLU_TRY(launch_lu_reg(kLuC64, crout, a, s, &launched));
  if (!launched) return clu_coop(crout, Y, ldy, R, C, perm, pub, sm_count(), status, first_zero, s);
  k_c_cm_to_rm_perm<<<tg, tb, 0, s>>>(X, ldx, R, C, perm, Y, ldy);
  return last_launch_status();
}

// Steps 1-2: d = exp(2 pi i theta) into d (n values), then Y = A D F S.
static int32_t srft_apply(const float* A, int64_t m, int64_t n, int64_t lda, const float* theta,
                          const int32_t* sel, int l, float2* d, const FftPlan& f, float2* Y,
                          int64_t ldy, int32_t* status, cudaStream_t s) {
  k_srft_phase<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(theta, (int)n, d);
  RLU_TRY(last_launch_status());
  const size_t fsmem = (size_t)n * sizeof(float2);
  const float scale = (float)(1.0 / std::sqrt((double)n));
  // the narrowest register array that holds n values over FFT_T threads
  auto go = [&](auto kern) -> int32_t {
    RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    kern<<<(unsigned)m, FFT_T, fsmem, s>>>(A, lda, (int)n, d, sel, l, scale, f, Y, ldy, status);
    return last_launch_status();
  };
  if (n <= FFT_T * 8) return go(k_srft_rows<8>);
  if (n <= FFT_T * 16) return go(k_srft_rows<16>);
  return go(k_srft_rows<FFT_MAXV>);
}

static int32_t fast_factor(const FastPlan& p, const float* A, int64_t m, int64_t n, int64_t lda,
                           int k, int l, const float* theta, const int32_t* sel, int32_t* P,
                           int32_t* Q, float2* L, int64_t ldl, float2* U, int64_t ldu,
                           rlu_info* info, char* ws, cudaStream_t s) {
  float2* d = reinterpret_cast<float2*>(ws + p.off_d);
  float2* Y = reinterpret_cast<float2*>(ws + p.off_Y);
  void* pub = ws + p.off_pub;
  float* S = reinterpret_cast<float*>(ws + p.off_S);
  double* V = reinterpret_cast<double*>(ws + p.off_V);
  double* Mre = reinterpret_cast<double*>(ws + p.off_M);
  float* Wst = reinterpret_cast<float*>(ws + p.off_Wst);
  float* AJ = reinterpret_cast<float*>(ws + p.off_AJ);
  float* Cst = reinterpret_cast<float*>(ws + p.off_C);
  float* Bst = reinterpret_cast<float*>(ws + p.off_B);
  float2* Bt = reinterpret_cast<float2*>(ws + p.off_Bt);
  float* Lbe = reinterpret_cast<float*>(ws + p.off_Lbe);
  float* Lo = reinterpret_cast<float*>(ws + p.off_Lo);
  int32_t* status = info ? &info->status : nullptr;
  const int k2 = 2 * k;
  if (info) RLU_TRY(info_init(info, s));
  // steps 1-2: Y = A D F S
  RLU_TRY(srft_apply(A, m, n, lda, theta, sel, l, d, p.fft, Y, l, status, s));
  // step 3: P Y = L_y U_y
  RLU_TRY(clu_factor(p, ws, false, Y, l, (int)m, l, P, pub, status,
                     info ? &info->nonfinite : nullptr,
                     info ? &info->first_zero_pivot_y : nullptr, s));
  // steps 4-6: V = L_y^H L_f (planes), M's real form, W = V L_1^{-1}, C = W A(J,:), B = M^{-1} C
  k_frlu_planes<<<dim3((unsigned)ceil_div(m, 32), (unsigned)ceil_div(l, 32)), dim3(32, 8), 0, s>>>(
      Y, l, (int)m, l, S);
  RLU_TRY(last_launch_status());
  if (p.tc) {  // V = S[:, :k]^T S: three TF32 products (A split on chip, S's parts), FP64 sum
    float* Sh = reinterpret_cast<float*>(ws + p.off_Sh);
    float* Sl = reinterpret_cast<float*>(ws + p.off_Sl);
    float* part2 = reinterpret_cast<float*>(ws + p.off_part2);
    RLU_TRY(split_parts(S, 2 * m, 2 * m, 2 * l, Sh, Sl, Bf16Parts{}, s));
    Umma3Op op{};
    op.A0 = S;
    op.lda = 2 * m;
    op.B0 = Sh;
    op.B1 = Sl;
    op.ldb = 2 * m;
    op.M = k;
    op.N = 2 * (int64_t)l;
    op.K = 2 * m;
    op.out = nullptr;
    op.splits = p.split_vt;
    op.partial = part2;
    op.status = status;
    RLU_TRY(umma3_gemm(U3_MODE_Y3, op, s));
    const int64_t kc = round_up(ceil_div(2 * m, p.split_vt), 32);
    RLU_TRY(splitk_reduce_f64(part2, (int)ceil_div(2 * m, kc), k, 2 * (int64_t)l, V,
                              2 * (int64_t)l, s));
  } else {
    GemmOp op{S, 2 * m, true, S, 2 * m, true, V, 2 * (int64_t)l, true, k, 2 * (int64_t)l, 2 * m,
              p.split_v, ws + p.off_part, false};
    RLU_TRY((gemm_simt<float, double>(op, s)));
  }
  k_frlu_embed<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)k2 * k2, 256), 4096), 256, 0, s>>>(
      V, 2 * (int64_t)l, k, l, Mre);
  RLU_TRY(last_launch_status());
  LdlOut<float> o{};
  o.LT = reinterpret_cast<float*>(ws + p.off_LT);
  o.LR = reinterpret_cast<float*>(ws + p.off_LR);
  o.W = reinterpret_cast<float*>(ws + p.off_W);
  o.WT = reinterpret_cast<float*>(ws + p.off_WT);
  o.dinv = reinterpret_cast<double*>(ws + p.off_dinv);
  o.k = k2;
  o.kp = p.kp;
  RLU_TRY(ldl_factor<float>(Mre, k2, o, status, s));
  {
    const int64_t ldv = 2 * (int64_t)l;
    int32_t st;
    switch (p.ns) {
      case 1: st = wsolve_launch<1>(V, ldv, k, l, Y, l, Wst, l, s); break;
      case 2: st = wsolve_launch<2>(V, ldv, k, l, Y, l, Wst, l, s); break;
      case 4: st = wsolve_launch<4>(V, ldv, k, l, Y, l, Wst, l, s); break;
      case 8: st = wsolve_launch<8>(V, ldv, k, l, Y, l, Wst, l, s); break;
      default: st = wsolve_launch<16>(V, ldv, k, l, Y, l, Wst, l, s); break;
    }
    RLU_TRY(st);
  }
  k_frlu_gather_aj<<<dim3((unsigned)std::min<int64_t>(ceil_div(n, 256), 64), (unsigned)l), 256, 0, s>>>(
      A, lda, (int)n, P, AJ, p.ldn);
  RLU_TRY(last_launch_status());
  if (p.tc) {  // C^T = A(J,:)^T W^T: A(J,:) as the raw n-contiguous operand, W's TF32 parts
    float* Wh = reinterpret_cast<float*>(ws + p.off_Wh);
    float* Wl = reinterpret_cast<float*>(ws + p.off_Wl);
    RLU_TRY(split_parts(Wst, l, l, k2, Wh, Wl, Bf16Parts{}, s));
    Umma3Op op{};
    op.A0 = AJ;
    op.lda = p.ldn;
    op.B0 = Wh;
    op.B1 = Wl;
    op.ldb = l;
    op.M = n;
    op.N = k2;
    op.K = l;
    op.out = Cst;
    op.ldo = p.ldn;
    op.out_colmajor = true;
    op.splits = umma3_splits(n, l, k2);
    op.partial = reinterpret_cast<float*>(ws + p.off_part2);
    op.status = status;
    RLU_TRY(umma3_gemm(U3_MODE_C3, op, s));
  } else {
    GemmOp op{Wst, l, true, AJ, p.ldn, false, Cst, p.ldn, true, k2, n, l, 1, nullptr, false};
    RLU_TRY((gemm_simt<float, float>(op, s)));
  }
  RLU_TRY(trsm_ldl<float>(o, Cst, p.ldn, n, Bst, p.ldn, s, ceil_div(n, 64) < sm_count()));
  // step 7: B Q = L_b U_b through the Crout LU of B^T
  k_frlu_pack_bt<<<dim3((unsigned)ceil_div(n, 32), (unsigned)ceil_div(k, 32)), dim3(32, 8), 0, s>>>(
      Bst, p.ldn, k, (int)n, Bt, k);
  RLU_TRY(last_launch_status());
  RLU_TRY(clu_factor(p, ws, true, Bt, k, (int)n, k, Q, pub, status,
                     info ? &info->nonfinite : nullptr,
                     info ? &info->first_zero_pivot_b : nullptr, s));
  // steps 8-9: U = U_b, L = L_y L_b
  k_frlu_unpack_u<<<dim3((unsigned)ceil_div(n, 32), (unsigned)ceil_div(k, 32)), dim3(32, 8), 0, s>>>(
      Bt, k, k, (int)n, U, ldu);
  RLU_TRY(last_launch_status());
  k_frlu_lb_embed<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)k * k, 256), 4096), 256, 0, s>>>(
      Bt, k, k, Lbe);
  RLU_TRY(last_launch_status());
  if (p.tc) {  // L's planes = S (read with ld m) Lbe: S as the raw m-contiguous operand
    float* Lbh = reinterpret_cast<float*>(ws + p.off_Lbh);
    float* Lbl = reinterpret_cast<float*>(ws + p.off_Lbl);
    // Lbe is row-major (row = K index); the operand wants its columns contiguous
    k_split_t<<<dim3((unsigned)ceil_div(k2, 32), (unsigned)ceil_div(k2, 32)), dim3(32, 8), 0, s>>>(
        Lbe, k2, k2, k2, Lbh, Lbl, k2);
    RLU_TRY(last_launch_status());
    Umma3Op op{};
    op.A0 = S;
    op.lda = m;
    op.B0 = Lbh;
    op.B1 = Lbl;
    op.ldb = k2;
    op.M = m;
    op.N = k2;
    op.K = k2;
    op.out = Lo;
    op.ldo = m;
    op.out_colmajor = true;
    op.splits = umma3_splits(m, k2, k2);
    op.partial = reinterpret_cast<float*>(ws + p.off_part2);
    op.status = status;
    RLU_TRY(umma3_gemm(U3_MODE_C3, op, s));
  } else {
    GemmOp op{S, m, false, Lbe, k2, false, Lo, m, false, m, k2, k2, 1, nullptr, false};
    RLU_TRY((gemm_simt<float, float>(op, s)));
  }
  k_frlu_pack_l<<<dim3((unsigned)std::min<int64_t>(ceil_div(m, 256), 64), (unsigned)k), 256, 0, s>>>(
      Lo, (int)m, k, L, ldl);
  return last_launch_status();
}

}  // namespace rlu

using namespace rlu;

extern "C" size_t rlu_fast_workspace_size(int64_t m, int64_t n, int32_t k, int32_t l) {
  FastPlan p;
  return fast_plan(m, n, k, l, p) == RLU_OK ? p.total : 0;
}

extern "C" size_t rlu_srft_workspace_size(int64_t n) {
  FftPlan f;
  if (n < 1 || n > (int64_t)FFT_T * FFT_MAXV || !fft_plan((int)n, f)) return 0;
  return (size_t)round_up(n * (int64_t)sizeof(float2), 256);
}

extern "C" int32_t rlu_srft_apply(const float* A, int64_t m, int64_t n, int64_t lda,
                                  const float* theta, const int32_t* s, int32_t l, void* Y,
                                  int64_t ldy, rlu_info* info, void* workspace, size_t ws_bytes,
                                  void* stream) {
  if (!A || !theta || !s || !Y) return RLU_EINVAL;
  if (m < 1 || n < 1 || l < 1 || l > n || lda < n || ldy < l) return RLU_EINVAL;
  if (m > INT_MAX) return RLU_EUNSUPPORTED;
  FftPlan f;
  if (n > (int64_t)FFT_T * FFT_MAXV || !fft_plan((int)n, f)) return RLU_EUNSUPPORTED;
  if (workspace == nullptr || ws_bytes < rlu_srft_workspace_size(n)) return RLU_ENOMEM;
  if (((uintptr_t)workspace & 255u) != 0) return RLU_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (info) RLU_TRY(info_init(info, st));
  return srft_apply(A, m, n, lda, theta, s, l, static_cast<float2*>(workspace), f,
                    static_cast<float2*>(Y), ldy, info ? &info->status : nullptr, st);
}

extern "C" int32_t rlu_fast_factor(const float* A, int64_t m, int64_t n, int64_t lda, int32_t k,
                                   int32_t l, const float* theta, const int32_t* s,
                                   int32_t* P, int32_t* Q, void* L, int64_t ldl, void* U,
                                   int64_t ldu, rlu_info* info, void* workspace,
                                   size_t ws_bytes, void* stream) {
  if (!A || !theta || !s || !P || !Q || !L || !U) return RLU_EINVAL;
  if (lda < n || ldl < m || ldu < n) return RLU_EINVAL;
  FastPlan p;
  RLU_TRY(fast_plan(m, n, k, l, p));
  if (workspace == nullptr || ws_bytes < p.total) return RLU_ENOMEM;
  if (((uintptr_t)workspace & 255u) != 0) return RLU_EINVAL;
  return fast_factor(p, A, m, n, lda, k, l, theta, s, P, Q, static_cast<float2*>(L), ldl,
                     static_cast<float2*>(U), ldu, info, static_cast<char*>(workspace),
                     static_cast<cudaStream_t>(stream));
}
