// Register-resident pivoted LU of a tall-skinny column-major X (R x C) on one thread-block
// cluster: the fast form of steps 3 (Doolittle, X = Y) and 6 (Crout, X = B^T) of
// Algorithm 1, with the same swap-free position bookkeeping and tie rule as panel_lu.cu
// (largest |value|, then smallest current position, which is getf2's choice).
//
// One launch factors one panel of up to NB-1 columns; the positions of the rows persist in
// global memory between launches, and k_lu_trail (all SMs) applies each panel's rank-w
// update to the remaining columns. Each thread owns RT rows; the panel's part of each row
// lives in registers and shifts by one register per step, so the rank-1 update is
// register-to-register. The
// per-step exchange avoids cluster barriers: every CTA reduces its candidates (warp
// reductions on order-preserving integer keys), stages one record (key, position, row,
// its pending multiplier and its row values) and pushes it with st.async into a receive
// slot of every CTA of the cluster, completing bytes on that CTA's mbarrier. Each CTA waits
// on its own mbarrier, picks the winner among the cluster's records and rebuilds the
// pivot row locally. Only the next column of each row is updated before the exchange; the
// rest of the update runs while the records are in flight (receivers apply the winner's
// pending update themselves).
//
// Waits on an mbarrier give up after about one second (globaltimer); the kernel then
// records RLU_ETIMEOUT in the status word and keeps going without waiting, so every CTA
// still reaches the same cluster barriers and exits.
#include <cooperative_groups.h>

#include "common.cuh"
#include "panel_lu.cuh"

namespace cg = cooperative_groups;

namespace rlu {

static constexpr int LR_NT = 512;
static constexpr int LR_NW = LR_NT / 32;
static constexpr int LR_CH = 32;  // trailing-update column chunk

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arm(uint32_t bar, uint32_t tx) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
               ::"r"(bar), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n"
               " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ void st_async16(uint32_t raddr, uint4 v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];\n"
               ::"r"(raddr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(rbar) : "memory");
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// Order-preserving 64-bit key of |v| (0 for NaN, so that a NaN never beats a number).
__device__ __forceinline__ uint64_t mag_key(float v) {
  const float a = fabsf(v);
  return (a == a) ? (uint64_t)__float_as_uint(a) : 0ull;
}
__device__ __forceinline__ uint64_t mag_key(double v) {
  const double a = fabs(v);
  return (a == a) ? (uint64_t)__double_as_longlong(a) : 0ull;
}

// Reciprocal of a pivot: correctly rounded in FP32; FP32 seed and two Newton steps in FP64
// (IEEE divide outside the FP32 exponent range). Multipliers are x * (1/pivot).
__device__ __forceinline__ float rcp_piv(float p) { return __frcp_rn(p); }
__device__ __forceinline__ double rcp_piv(double p) {
  const double a = fabs(p);
  if (!(a > 1e-30 && a < 1e30)) return 1.0 / p;
  double y = (double)__frcp_rn((float)p);
  double e = fma(-p, y, 1.0);
  y = fma(y, e, y);
  e = fma(-p, y, 1.0);
  return fma(y, e, y);
}

// Warp-wide winner: largest key, then smallest position; returns the winning lane.
__device__ __forceinline__ int warp_winner(uint64_t key, int pos) {
  const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
  const uint32_t mhi = __reduce_max_sync(0xffffffffu, hi);
  const uint32_t mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  const bool top = (hi == mhi) && (lo == mlo);
  const int mpos = (int)__reduce_min_sync(0xffffffffu, top ? (uint32_t)pos : 0x7fffffffu);
  const uint32_t who = __ballot_sync(0xffffffffu, top && pos == mpos);
  return __ffs(who) - 1;
}

// Vector shared-memory access of 4 consecutive elements (16-byte aligned for float).
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
  *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
}

template <int NB>
struct Pad4 { static constexpr int value = (NB + 3) / 4 * 4; };

template <typename T, int NB>
struct LrRec {  // one candidate record, 16-byte chunks
  uint32_t khi, klo;
  int32_t pos, row;
  T xe;       // the candidate's value in the current column
  T mp;       // its pending multiplier of the previous step (0 at a panel start)
  alignas(16) T x[Pad4<NB>::value];  // its registers (previous shift)
};

template <typename T, int NB>
__host__ __device__ constexpr int rec_bytes() { return (int)((sizeof(LrRec<T, NB>) + 15) / 16 * 16); }

template <typename T, int NB>
struct LrShared {
  uint64_t mbar[2];
  int32_t err;
  int32_t nonfinite;
  uint32_t wkhi[LR_NW], wklo[LR_NW];
  int32_t wpos[LR_NW], wrow[LR_NW];
  alignas(16) unsigned char stage[rec_bytes<T, NB>()];
  alignas(16) unsigned char recv[2][16][rec_bytes<T, NB>()];
  T pval[2];                               // pivot value of the step of that parity
  alignas(16) T prow[2][Pad4<NB>::value + 4];  // P1[c] = pivot row at offset c + 1
};

template <typename T, bool CROUT, int RT, int NB>
__global__ void __launch_bounds__(LR_NT, 1) k_lu_reg(LuArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int ncta = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rpc = a.rpc;  // = LR_NT * RT (rows per CTA)
  const int r0 = crank * rpc;
  const int C = a.C, R = a.R;
  const int64_t ldx = a.ldx;
  T* __restrict__ X = static_cast<T*>(a.X);
  constexpr int RB = rec_bytes<T, NB>();
  constexpr int NCHUNK = RB / 16;
  static_assert(NCHUNK <= 32, "record must fit one warp's 16-byte chunks");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  LrShared<T, NB>& sh = *reinterpret_cast<LrShared<T, NB>*>(smem_raw);
  size_t off = (sizeof(LrShared<T, NB>) + 15) / 16 * 16;
  T* L11 = reinterpret_cast<T*>(smem_raw + off);          // [NB][NB]
  off += (sizeof(T) * (size_t)NB * NB + 15) / 16 * 16;
  int* psmall = reinterpret_cast<int*>(smem_raw + off);   // [C]

  // rows of this thread: r0 + tid + s*LR_NT
  int rowi[RT];
  int pos[RT];
  bool have[RT];
  const bool first = (a.p0 == 0);
#pragma unroll
  for (int s = 0; s < RT; ++s) {
    rowi[s] = r0 + tid + s * LR_NT;
    have[s] = (tid + s * LR_NT < rpc) && rowi[s] < R;
    pos[s] = (first || !have[s]) ? rowi[s] : a.posg[rowi[s]];
  }
  for (int p = tid; p < C; p += LR_NT) psmall[p] = first ? p : a.psg[p];
  if (tid == 0) {
    mbar_init(smem_u32(&sh.mbar[0]), 1);
    mbar_init(smem_u32(&sh.mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    sh.err = 0;
    sh.nonfinite = 0;
  }
  for (int i = tid; i < 2 * (Pad4<NB>::value + 4); i += LR_NT) (&sh.prow[0][0])[i] = T(0);
  cl.sync();

  const uint32_t stage_a = smem_u32(sh.stage);
  const uint32_t recv_a = smem_u32(&sh.recv[0][0][0]);
  const uint32_t mbar_a = smem_u32(&sh.mbar[0]);
  int first_zero = -1;
  bool timed_out = false;

  T x[RT][NB];
  T xe[RT], mp[RT];

  {
    const int p0 = a.p0;
    const int w = a.pw;
    // load: x[s][c] = X[p0 - 1 + c] for c = 1..w (x[s][0] unused), pending multiplier 0
#pragma unroll
    for (int s = 0; s < RT; ++s) {
      x[s][0] = T(0);
#pragma unroll
      for (int c = 1; c < NB; ++c)
        x[s][c] = (have[s] && c <= w) ? X[(int64_t)(p0 - 1 + c) * ldx + rowi[s]] : T(0);
      xe[s] = x[s][1];
      mp[s] = T(0);
    }
    for (int i = tid; i < Pad4<NB>::value + 4; i += LR_NT) {
      sh.prow[0][i] = T(0);
      sh.prow[1][i] = T(0);
    }
    __syncthreads();

    for (int jj = 0; jj < w; ++jj) {
      const int j = p0 + jj;
      const int par = j & 1;
      const int a_row = psmall[j];
      if (tid == 0) mbar_arm(mbar_a + 8 * par, (uint32_t)(ncta * RB));
      // ---- candidates: thread, warp, CTA ------------------------------------------------
      uint64_t key = 0;
      int kpos = 0x7fffffff, ks = 0;
      bool anyc = false;
#pragma unroll
      for (int s = 0; s < RT; ++s) {
        if (have[s] && pos[s] >= j) {
          if (!is_finite_val(xe[s])) sh.nonfinite = 1;
          const uint64_t kk = mag_key(xe[s]);
          if (!anyc || kk > key || (kk == key && pos[s] < kpos)) {
            key = kk;
            kpos = pos[s];
            ks = s;
          }
          anyc = true;
        }
      }
      int krow = anyc ? rowi[ks] : -1;
      if (!anyc) key = 0;
      {
        // empty candidates lose to every real one: give them the largest position
        const int wl = warp_winner(anyc ? key : 0ull, anyc ? kpos : 0x7fffffff);
        const uint64_t wk = __shfl_sync(0xffffffffu, key, wl);
        const int wp = __shfl_sync(0xffffffffu, anyc ? kpos : 0x7fffffff, wl);
        const int wr = __shfl_sync(0xffffffffu, krow, wl);
        if (lane == 0) {
          sh.wkhi[warp] = (uint32_t)(wk >> 32);
          sh.wklo[warp] = (uint32_t)wk;
          sh.wpos[warp] = wp;
          sh.wrow[warp] = wr;
        }
      }
      __syncthreads();
      int cta_row, cta_pos;
      uint64_t cta_key;
      {
        const uint64_t k2 = lane < LR_NW ? (((uint64_t)sh.wkhi[lane] << 32) | sh.wklo[lane]) : 0ull;
        const int p2 = lane < LR_NW ? sh.wpos[lane] : 0x7fffffff;
        const int wl = warp_winner(k2, p2);
        cta_key = __shfl_sync(0xffffffffu, k2, wl);
        cta_pos = __shfl_sync(0xffffffffu, p2, wl);
        cta_row = sh.wrow[wl < LR_NW ? wl : 0];
      }
      // the thread that owns the CTA's candidate stages its record
#pragma unroll
      for (int s = 0; s < RT; ++s) {
        if (have[s] && rowi[s] == cta_row) {
          LrRec<T, NB>* rec = reinterpret_cast<LrRec<T, NB>*>(sh.stage);
          rec->khi = (uint32_t)(cta_key >> 32);
          rec->klo = (uint32_t)cta_key;
          rec->pos = cta_pos;
          rec->row = cta_row;
          rec->xe = xe[s];
          rec->mp = mp[s];
#pragma unroll
          for (int c = 0; c + 3 < NB; c += 4)
            st4(&rec->x[c], x[s][c], x[s][c + 1], x[s][c + 2], x[s][c + 3]);
#pragma unroll
          for (int c = NB / 4 * 4; c < NB; ++c) rec->x[c] = x[s][c];
        }
      }
      if (cta_row < 0 && tid == 0) {  // no live row in this CTA
        LrRec<T, NB>* rec = reinterpret_cast<LrRec<T, NB>*>(sh.stage);
        rec->khi = 0;
        rec->klo = 0;
        rec->pos = 0x7fffffff;
        rec->row = -1;
        rec->xe = T(0);
        rec->mp = T(0);
      }
      __syncthreads();
      // ---- push the record to every CTA (warp w -> CTA w) ------------------------------
      if (warp < ncta && lane < NCHUNK) {
        const uint4 v = *reinterpret_cast<const uint4*>(sh.stage + 16 * lane);
        const uint32_t dst = map_rank(recv_a + (uint32_t)((par * 16 + crank) * RB + 16 * lane), warp);
        const uint32_t bar = map_rank(mbar_a + 8 * par, warp);
        st_async16(dst, v, bar);
      }
      // ---- meanwhile: the deferred part of the previous step's update ------------------
      if (jj > 0) {
        const T* P1 = sh.prow[par ^ 1];  // P1[c] = previous pivot row at offset c + 1
#pragma unroll
        for (int c0 = 0; c0 < NB - 1; c0 += 4) {
          T pv[4];
          ld4(P1 + c0, pv);
#pragma unroll
          for (int s = 0; s < RT; ++s) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (c0 + u < NB - 1) x[s][c0 + u] = fma(-mp[s], pv[u], x[s][c0 + u + 1]);
          }
        }
#pragma unroll
        for (int s = 0; s < RT; ++s) x[s][NB - 1] = T(0);
      } else {
#pragma unroll
        for (int s = 0; s < RT; ++s) {
#pragma unroll
          for (int c = 0; c < NB - 1; ++c) x[s][c] = x[s][c + 1];
          x[s][NB - 1] = T(0);
        }
      }
      // ---- wait for the cluster's records -----------------------------------------------
      if (!timed_out) {
        const uint32_t bar = mbar_a + 8 * par;
        const uint32_t ph = (uint32_t)((j >> 1) & 1);
        if (!mbar_try(bar, ph)) {
          const uint64_t t0 = gtimer();
          while (!mbar_try(bar, ph)) {
            if (gtimer() - t0 > 1000000000ull) {
              timed_out = true;
              sh.err = 1;
              break;
            }
          }
        }
      }
      // ---- winner among the cluster's records --------------------------------------------
      int win;
      {
        const LrRec<T, NB>* rr = reinterpret_cast<const LrRec<T, NB>*>(&sh.recv[par][lane < ncta ? lane : 0][0]);
        const uint64_t k3 = lane < ncta ? (((uint64_t)rr->khi << 32) | rr->klo) : 0ull;
        const int p3 = lane < ncta ? rr->pos : 0x7fffffff;
        win = warp_winner(k3, p3);
      }
      const LrRec<T, NB>* W = reinterpret_cast<const LrRec<T, NB>*>(&sh.recv[par][win][0]);
      const int wrow = W->row, wpos = W->pos;
      const bool valid = wrow >= 0;
      const T piv = W->xe;
      const bool nz = valid && piv != T(0) && mag_key(piv) != 0ull;
      const T rp = nz ? rcp_piv(piv) : T(0);
      // pivot row: value P_j[0] = piv and P1_j[c] = P_j[c + 1] (column j + 1 + c), from
      // the winner's registers and its pending update
      {
        const T* Pp = sh.prow[par ^ 1];
        T* Pn1 = sh.prow[par];
        const T wm = W->mp;
        for (int c = tid; c < Pad4<NB>::value + 4; c += LR_NT) {
          T v = T(0);
          if (c + 1 < w - jj) {  // column j + 1 + c lies in the panel
            v = (wm != T(0)) ? fma(-wm, Pp[c + 1], W->x[c + 2]) : W->x[c + 2];
            if (CROUT && nz) v = v * rp;
          }
          Pn1[c] = v;
        }
        if (tid == 0) sh.pval[par] = piv;
      }
      if (tid == 0) {
        if (valid && wrow != a_row) {
          psmall[j] = wrow;
          if (wpos < C) psmall[wpos] = a_row;
        }
        if (!nz && first_zero < 0) first_zero = j;
      }
      __syncthreads();
      // positions of my rows after the swap of positions j and wpos
      if (valid && wrow != a_row) {
#pragma unroll
        for (int s = 0; s < RT; ++s) {
          if (rowi[s] == a_row) pos[s] = wpos;
          if (rowi[s] == wrow) pos[s] = j;
        }
      }
      const T* Pn1 = sh.prow[par];
      // the pivot row's final entries: columns j .. p0 + w - 1
      if (valid && wrow >= r0 && wrow < r0 + rpc) {
        for (int c = tid; c < w - jj; c += LR_NT)
          X[(int64_t)(j + c) * ldx + wrow] = (c == 0) ? piv : Pn1[c - 1];
      }
      // multipliers of my live rows, and the eager update of the next column
#pragma unroll
      for (int s = 0; s < RT; ++s) {
        T m = T(0);
        if (have[s] && pos[s] > j && nz) {
          m = CROUT ? xe[s] : xe[s] * rp;
          X[(int64_t)j * ldx + rowi[s]] = m;
        } else if (have[s] && pos[s] > j) {
          // zero pivot: nothing is eliminated; the column keeps its (zero) values
          X[(int64_t)j * ldx + rowi[s]] = xe[s];
        }
        mp[s] = m;
        xe[s] = (m != T(0)) ? fma(-m, Pn1[0], x[s][1]) : x[s][1];
      }
    }

    // all records of this panel consumed before anyone reuses receive slots / exits
    cl.sync();
    if (p0 + w < C) {
      // ---- U12 of the pivot rows for the trailing columns (forward substitution) -------
      for (int e = tid; e < w * w; e += LR_NT) {
        const int t = e / w, s = e % w;
        L11[t * NB + s] = X[(int64_t)(p0 + s) * ldx + psmall[p0 + t]];
      }
      __syncthreads();
      for (int c = p0 + w + crank * LR_NW + warp; c < C; c += ncta * LR_NW) {
        constexpr int NQ = (NB + 31) / 32;
        T u[NQ], fin[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int t = lane + 32 * q;
          u[q] = t < w ? X[(int64_t)c * ldx + psmall[p0 + t]] : T(0);
          fin[q] = u[q];
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          for (int s = 32 * q; s < min(w, 32 * q + 32); ++s) {
            T us = __shfl_sync(0xffffffffu, u[q], s - 32 * q);
            if (CROUT) {
              const T pv = L11[s * NB + s];
              if (pv != T(0)) us = us * rcp_piv(pv);
            }
            if (lane == s - 32 * q) fin[q] = us;
#pragma unroll
            for (int qq = q; qq < NQ; ++qq) {
              const int t = lane + 32 * qq;
              if (t > s && t < w) u[qq] = fma(-L11[t * NB + s], us, u[qq]);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int t = lane + 32 * q;
          if (t < w) X[(int64_t)c * ldx + psmall[p0 + t]] = fin[q];
        }
      }
    }
  }

  // persist the positions for the next panel; the last panel writes P (gather form)
  const bool last = (a.p0 + a.pw >= C);
#pragma unroll
  for (int s = 0; s < RT; ++s)
    if (have[s]) a.posg[rowi[s]] = pos[s];
  if (crank == 0)
    for (int p = tid; p < C; p += LR_NT) a.psg[p] = psmall[p];
  if (last) {
#pragma unroll
    for (int s = 0; s < RT; ++s)
      if (have[s]) a.perm[pos[s]] = rowi[s];
  }
  if (tid == 0) {
    if (crank == 0 && a.zero_step && first_zero >= 0) atomicCAS(a.zero_step, -1, first_zero);
    if (sh.nonfinite && a.nonfinite) atomicOr(a.nonfinite, 1);
    if (sh.err && a.status) atomicExch(a.status, RLU_ETIMEOUT);
  }
  cl.sync();
}

// Rank-w update of the trailing columns [c_begin, C) of every row whose position is at
// least p0 + w: X[r][c] -= sum_s X[r][p0+s] * U12[s][c], U12 = the panel's pivot rows
// (already solved by the panel launch). One thread per row, 32 columns per CTA.
template <typename T>
__global__ void __launch_bounds__(256) k_lu_trail(T* __restrict__ X, int64_t ldx, int R, int C,
                                                 int p0, int w, const int32_t* __restrict__ posg,
                                                 const int32_t* __restrict__ psg) {
  __shared__ __align__(16) T U12[128][LR_CH];
  const int c0 = p0 + w + blockIdx.y * LR_CH;
  const int cw = min(LR_CH, C - c0);
  for (int e = threadIdx.x; e < w * LR_CH; e += 256) {
    const int s = e / LR_CH, q = e % LR_CH;
    U12[s][q] = q < cw ? X[(int64_t)(c0 + q) * ldx + psg[p0 + s]] : T(0);
  }
  __syncthreads();
  const int r = blockIdx.x * 256 + threadIdx.x;
  if (r >= R || posg[r] < p0 + w) return;
  T acc[LR_CH];
#pragma unroll
  for (int q = 0; q < LR_CH; ++q) acc[q] = q < cw ? X[(int64_t)(c0 + q) * ldx + r] : T(0);
  for (int s = 0; s < w; ++s) {
    const T lv = X[(int64_t)(p0 + s) * ldx + r];
#pragma unroll
    for (int q = 0; q < LR_CH; q += 4) {
      T uv[4];
      ld4(&U12[s][q], uv);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[q + u] = fma(-lv, uv[u], acc[q + u]);
    }
  }
#pragma unroll
  for (int q = 0; q < LR_CH; ++q)
    if (q < cw) X[(int64_t)(c0 + q) * ldx + r] = acc[q];
}

template <typename T, int NB>
static size_t lr_smem_bytes(int rpc, int C) {
  size_t b = (sizeof(LrShared<T, NB>) + 15) / 16 * 16;
  b += (sizeof(T) * (size_t)NB * NB + 15) / 16 * 16;
  b += sizeof(int) * (size_t)C;
  (void)rpc;
  return b;
}

template <typename T, bool CROUT, int RT, int NB>
static int32_t try_launch(const LuArgs& in, cudaStream_t s, bool* launched) {
  *launched = false;
  const int rpc = LR_NT * RT;
  const int ncta = (int)ceil_div(in.R, rpc);
  if (ncta > 16) return RLU_OK;
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t bytes = lr_smem_bytes<T, NB>(rpc, in.C);
  if (bytes > (size_t)optin) return RLU_OK;
  auto kern = k_lu_reg<T, CROUT, RT, NB>;
  RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(ncta);
  cfg.blockDim = dim3(LR_NT);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (ncta > 8) {
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      return RLU_OK;
    }
  }
  if (!in.posg || !in.psg) return RLU_OK;  // no position state: use the one-launch kernel
  LuArgs a = in;
  a.rpc = rpc;
  a.nb = NB - 1;
  for (int p0 = 0; p0 < in.C; p0 += NB - 1) {
    a.p0 = p0;
    a.pw = min(NB - 1, in.C - p0);
    RLU_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
    RLU_TRY(last_launch_status());
    *launched = true;
    if (p0 + a.pw < in.C) {
      const dim3 grid((unsigned)ceil_div(in.R, 256), (unsigned)ceil_div(in.C - p0 - a.pw, LR_CH));
      k_lu_trail<T><<<grid, 256, 0, s>>>(static_cast<T*>(in.X), in.ldx, in.R, in.C, p0, a.pw,
                                         in.posg, in.psg);
      RLU_TRY(last_launch_status());
    }
  }
  return RLU_OK;
}

template <typename T, bool CROUT>
static int32_t launch_reg_t(const LuArgs& a, cudaStream_t s, bool* launched) {
  // rows per thread RT and register panel NB (NB - 1 columns per panel)
  constexpr int W1 = sizeof(T) == 4 ? 77 : 37;
  constexpr int W2 = sizeof(T) == 4 ? 37 : 19;
  constexpr int W4 = sizeof(T) == 4 ? 17 : 9;
  if (a.R <= 16 * LR_NT) RLU_TRY((try_launch<T, CROUT, 1, W1>(a, s, launched)));
  if (!*launched && a.R <= 32 * LR_NT) RLU_TRY((try_launch<T, CROUT, 2, W2>(a, s, launched)));
  if (!*launched && a.R <= 64 * LR_NT) RLU_TRY((try_launch<T, CROUT, 4, W4>(a, s, launched)));
  return RLU_OK;
}

int32_t launch_lu_reg(int32_t dtype, bool crout, const LuArgs& a, cudaStream_t s, bool* launched) {
  *launched = false;
  if (dtype == RLU_F64) return crout ? launch_reg_t<double, true>(a, s, launched) : launch_reg_t<double, false>(a, s, launched);
  if (dtype == RLU_F32) return crout ? launch_reg_t<float, true>(a, s, launched) : launch_reg_t<float, false>(a, s, launched);
  return RLU_OK;
}

}  // namespace rlu
