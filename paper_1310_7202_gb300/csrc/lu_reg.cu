// Register-resident pivoted LU of a tall-skinny column-major X (R x C) on one thread-block
// cluster: the fast form of steps 3 (Doolittle, X = Y) and 6 (Crout, X = B^T) of
// Algorithm 1, with the same swap-free position bookkeeping and tie rule as panel_lu.cu
// (largest |value|, then smallest current position, which is getf2's choice). The element
// type is float, double or cf32 (complex FP32, for the fast randomized LU of Algorithm 4,
// whose pivots go by |Re| + |Im|).
//
// One launch factors one panel of up to NB-1 columns; the positions of the rows persist in
// global memory between launches, and k_lu_trail (all SMs) applies each panel's rank-w
// update to the remaining columns. Narrow panels (tall X, several rows per thread) are
// grouped into blocks of about 64 columns, a right-looking blocked LU: a panel's update
// reaches only the rest of its block, and each block's pivot rows are solved (k_lu_u12)
// and its rank-64 update applied to the columns after the block once, so that the
// trailing columns are read and written once per block rather than once per panel. Each thread owns RT rows; the panel's part of each row
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
// A problem whose rows fit one CTA (SOLO) skips the exchange: the owner warp writes its
// record straight into the receive slot, a CTA barrier after the deferred update publishes
// it, and that record is the winner.
//
// Waits on an mbarrier give up after about one second (globaltimer); the kernel then
// records RLU_ETIMEOUT in the status word and keeps going without waiting, so every CTA
// still reaches the same cluster barriers and exits.
#include <cooperative_groups.h>
#include <type_traits>

#include "common.cuh"
#include "panel_lu.cuh"
#include "umma.cuh"

namespace cg = cooperative_groups;

namespace rlu {

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
// Test for completion of the phase of the given parity; the warp may sleep in the
// instruction up to the hinted time (ns) instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n"
               " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
               " selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(bar), "r"(parity), "r"(20000u) : "memory");
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
  return (a == a) ? ((uint64_t)__float_as_uint(a) << 32) : 0ull;
}
__device__ __forceinline__ uint64_t mag_key(double v) {
  const double a = fabs(v);
  return (a == a) ? (uint64_t)__double_as_longlong(a) : 0ull;
}
// Complex FP32 (the fast randomized LU of Algorithm 4): pivots by |Re| + |Im|.
__device__ __forceinline__ uint64_t mag_key(cf32 v) {
  const float a = fabsf(v.x) + fabsf(v.y);
  return (a == a) ? ((uint64_t)__float_as_uint(a) << 32) : 0ull;
}

// Reciprocal of a pivot: the hardware approximation refined by Newton-Raphson steps
// (y' = y + y (1 - p y)): one step in FP32 (within an ulp or so), two from the FP32 seed in
// FP64 (IEEE divide outside the FP32 exponent range). Multipliers are x * (1/pivot).
__device__ __forceinline__ float rcp_approx(float p) {
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(p));
  return y;
}
__device__ __forceinline__ float rcp_piv(float p) {
  const float y = rcp_approx(p);
  if (!isfinite(y)) return y;
  return fmaf(y, fmaf(-p, y, 1.0f), y);
}
// 1 / p with the larger of |Re p|, |Im p| scaled out first (no overflow of |p|^2)
__device__ __forceinline__ cf32 rcp_piv(cf32 p) {
  const float sc = fmaxf(fabsf(p.x), fabsf(p.y));
  const float qx = p.x / sc, qy = p.y / sc;
  const float den = (qx * qx + qy * qy) * sc;
  return cf32(qx / den, -qy / den);
}
__device__ __forceinline__ double rcp_piv(double p) {
  const double a = fabs(p);
  if (!(a > 1e-30 && a < 1e30)) return 1.0 / p;
  double y = (double)rcp_approx((float)p);
  double e = fma(-p, y, 1.0);
  y = fma(y, e, y);
  e = fma(-p, y, 1.0);
  return fma(y, e, y);
}

// Warp-wide winner: largest key, then smallest position; returns the winning lane. The
// common case (one lane holds the largest high word) costs one reduction and one ballot.
__device__ __forceinline__ int warp_winner(uint64_t key, int pos) {
  const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
  const uint32_t mhi = __reduce_max_sync(0xffffffffu, hi);
  bool top = hi == mhi;
  uint32_t who = __ballot_sync(0xffffffffu, top);
  if (__popc(who) > 1) {
    const uint32_t mlo = __reduce_max_sync(0xffffffffu, top ? lo : 0u);
    top = top && lo == mlo;
    who = __ballot_sync(0xffffffffu, top);
    if (__popc(who) > 1) {
      const int mpos = (int)__reduce_min_sync(0xffffffffu, top ? (uint32_t)pos : 0x7fffffffu);
      who = __ballot_sync(0xffffffffu, top && pos == mpos);
    }
  }
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
__device__ __forceinline__ void ld4(const cf32* p, cf32 (&o)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 2);
  o[0] = cf32(a.x, a.y); o[1] = cf32(a.z, a.w); o[2] = cf32(b.x, b.y); o[3] = cf32(b.z, b.w);
}
__device__ __forceinline__ void st4(cf32* p, cf32 a, cf32 b, cf32 c, cf32 d) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  *reinterpret_cast<float4*>(p + 2) = make_float4(c.x, c.y, d.x, d.y);
}
// warp shuffle of one element
__device__ __forceinline__ float shfl_t(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_t(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ cf32 shfl_t(cf32 v, int src) {
  return cf32(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
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

template <typename T, int NB, int NW>
struct LrShared {
  uint64_t mbar[2];
  int32_t err;
  int32_t nonfinite;
  uint32_t wkhi[2][NW], wklo[2][NW];  // per-warp candidates, by step parity
  int32_t wpos[2][NW], wrow[2][NW];
  alignas(16) unsigned char stage[rec_bytes<T, NB>()];
  alignas(16) unsigned char recv[2][16][rec_bytes<T, NB>()];
  // per-warp copies of the pivot row, by step parity: P1[c] = pivot row at offset c + 1
  alignas(16) T prow[NW][2][Pad4<NB>::value + 4];
};

template <typename T, bool CROUT, int RT, int NB, int NT, bool SOLO>
__device__ __forceinline__ void lu_reg_body(const LuArgs& a) {
  constexpr int NW = NT / 32;
  cg::cluster_group cl = cg::this_cluster();
  const int ncta = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rpc = a.rpc;  // = NT * RT (rows per CTA)
  const int r0 = crank * rpc;
  const int C = a.C, R = a.R;
  const int64_t ldx = a.ldx;
  T* __restrict__ X = static_cast<T*>(a.X);
  constexpr int RB = rec_bytes<T, NB>();
  constexpr int NCHUNK = RB / 16;
  constexpr int PW = Pad4<NB>::value + 4;
  static_assert(NCHUNK <= 32, "record must fit one warp's 16-byte chunks");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  LrShared<T, NB, NW>& sh = *reinterpret_cast<LrShared<T, NB, NW>*>(smem_raw);
  size_t off = (sizeof(LrShared<T, NB, NW>) + 15) / 16 * 16;
  T* L11 = reinterpret_cast<T*>(smem_raw + off);          // [NB][NB]
  off += (sizeof(T) * (size_t)NB * NB + 15) / 16 * 16;
  int* prows = reinterpret_cast<int*>(smem_raw + off);    // [NB] this panel's pivot rows

  // rows of this thread: r0 + tid + s*NT
  int rowi[RT];
  int pos[RT];
  bool have[RT];
  const bool first = (a.p0 == 0);
#pragma unroll
  for (int s = 0; s < RT; ++s) {
    rowi[s] = r0 + tid + s * NT;
    have[s] = (tid + s * NT < rpc) && rowi[s] < R;
    pos[s] = (first || !have[s]) ? rowi[s] : a.posg[rowi[s]];
  }
  if (tid == 0) {
    mbar_init(smem_u32(&sh.mbar[0]), 1);
    mbar_init(smem_u32(&sh.mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    sh.err = 0;
    sh.nonfinite = 0;
  }
  for (int i = tid; i < NW * 2 * PW; i += NT) (&sh.prow[0][0][0])[i] = T(0);
  cl.sync();

  const uint32_t recv_a = smem_u32(&sh.recv[0][0][0]);
  const uint32_t mbar_a = smem_u32(&sh.mbar[0]);
  int first_zero = -1;
  bool timed_out = false;

  T x[RT][NB];
  T xe[RT], mp[RT];
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

  for (int jj = 0; jj < w; ++jj) {
    const int j = p0 + jj;
    // receive slots and mbarriers alternate by the step's parity within this launch; the
    // mbarriers start at phase 0 in every launch, so step jj waits on phase (jj / 2) & 1
    const int par = jj & 1;
    const int live = w - jj;  // columns j .. p0 + w - 1
    if (!SOLO && tid == 0) mbar_arm(mbar_a + 8 * par, (uint32_t)(ncta * RB));
    // ---- candidates: thread, warp ----------------------------------------------------------
    uint64_t key = 0;
    int kpos = 0x7fffffff, krow = -1;
#pragma unroll
    for (int s = 0; s < RT; ++s) {
      if (have[s] && pos[s] >= j) {
        if (!is_finite_val(xe[s])) sh.nonfinite = 1;
        const uint64_t kk = mag_key(xe[s]);
        if (krow < 0 || kk > key || (kk == key && pos[s] < kpos)) {
          key = kk;
          kpos = pos[s];
          krow = rowi[s];
        }
      }
    }
    {
      // empty candidates lose to every real one: key 0 and the largest position
      const int wl = warp_winner(key, kpos);
      if (lane == wl) {
        sh.wkhi[par][warp] = (uint32_t)(key >> 32);
        sh.wklo[par][warp] = (uint32_t)key;
        sh.wpos[par][warp] = kpos;
        sh.wrow[par][warp] = krow;
      }
    }
    __syncthreads();
    // ---- CTA winner, in every warp; its warp stages the record and pushes it -------------
    {
      const uint64_t k2 = lane < NW ? (((uint64_t)sh.wkhi[par][lane] << 32) | sh.wklo[par][lane]) : 0ull;
      const int p2 = lane < NW ? sh.wpos[par][lane] : 0x7fffffff;
      const int ow = warp_winner(k2, p2);  // owner warp
      if (warp == ow) {
        const int cta_row = sh.wrow[par][ow];
        LrRec<T, NB>* rec = reinterpret_cast<LrRec<T, NB>*>(SOLO ? &sh.recv[par][0][0] : sh.stage);
        if (cta_row < 0) {
          if (lane == 0) {  // no live row in this CTA
            rec->khi = 0;
            rec->klo = 0;
            rec->pos = 0x7fffffff;
            rec->row = -1;
            rec->xe = T(0);
            rec->mp = T(0);
          }
        } else {
#pragma unroll
          for (int s = 0; s < RT; ++s) {
            if (have[s] && rowi[s] == cta_row) {
              rec->khi = sh.wkhi[par][ow];
              rec->klo = sh.wklo[par][ow];
              rec->pos = sh.wpos[par][ow];
              rec->row = cta_row;
              rec->xe = xe[s];
              rec->mp = mp[s];
#pragma unroll
              for (int c = 0; c + 3 < NB; c += 4)
                if (c < live + 2) st4(&rec->x[c], x[s][c], x[s][c + 1], x[s][c + 2], x[s][c + 3]);
#pragma unroll
              for (int c = NB / 4 * 4; c < NB; ++c) rec->x[c] = x[s][c];
            }
          }
        }
        __syncwarp();
        if (!SOLO && lane < NCHUNK) {
          const uint4 v = *reinterpret_cast<const uint4*>(sh.stage + 16 * lane);
          const uint32_t dst = recv_a + (uint32_t)((par * 16 + crank) * RB + 16 * lane);
          const uint32_t bar = mbar_a + 8 * par;
          for (int r = 0; r < ncta; ++r) st_async16(map_rank(dst, r), v, map_rank(bar, r));
        }
      }
    }
    // ---- meanwhile: the deferred part of the previous step's update --------------------------
    if (jj > 0) {
      const T* P1 = sh.prow[warp][par ^ 1];  // P1[c] = previous pivot row at offset c + 1
      // FP32: every block of the panel, also those past the live columns (their registers
      // are never read again): skipping them behind a branch costs more instructions
      // (register moves at the join) than their multiply-adds. FP64 multiply-adds are slow
      // enough that the blocks past the live columns are skipped.
      constexpr bool kAllBlocks = sizeof(T) == 4;
#pragma unroll
      for (int b0 = 0; b0 < NB - 1; b0 += 16) {
        if (kAllBlocks || b0 < live) {
#pragma unroll
          for (int c0 = b0; c0 < b0 + 16 && c0 < NB - 1; c0 += 4) {
            T pv[4];
            ld4(P1 + c0, pv);
#pragma unroll
            for (int s = 0; s < RT; ++s) {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (c0 + u < NB - 1) x[s][c0 + u] = fma(-mp[s], pv[u], x[s][c0 + u + 1]);
            }
          }
        }
      }
    } else {
#pragma unroll
      for (int s = 0; s < RT; ++s) {
#pragma unroll
        for (int c = 0; c < NB - 1; ++c) x[s][c] = x[s][c + 1];
        x[s][NB - 1] = T(0);
      }
    }
    // ---- wait for the cluster's records -----------------------------------------------------
    if (SOLO) {
      __syncthreads();  // the owner warp's record in slot 0
    } else if (!timed_out) {
      const uint32_t bar = mbar_a + 8 * par;
      const uint32_t ph = (uint32_t)((jj >> 1) & 1);
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
    // ---- winner among the cluster's records, in every warp ----------------------------------
    int win = 0;
    if (!SOLO) {
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
    // this warp's copy of the pivot row: P1_j[c] = column j + 1 + c, from the winner's
    // registers and its pending update
    T* Pn1 = sh.prow[warp][par];
    {
      const T* Pp = sh.prow[warp][par ^ 1];
      const T wm = W->mp;
      // live entries only (c + 1 < live); the entries past them are stale and reach only
      // registers of columns that have left the panel
      for (int c = lane; c + 1 < live; c += 32) {
        T v = (wm != T(0)) ? fma(-wm, Pp[c + 1], W->x[c + 2]) : W->x[c + 2];
        if (CROUT && nz) v = v * rp;
        Pn1[c] = v;
      }
    }
    __syncwarp();
    if (tid == 0) {
      prows[jj] = valid ? wrow : -1;
      if (!nz && first_zero < 0) first_zero = j;
    }
    // positions of my rows after the exchange of positions j and wpos
    if (valid) {
#pragma unroll
      for (int s = 0; s < RT; ++s) {
        if (rowi[s] == wrow) pos[s] = j;
        else if (pos[s] == j) pos[s] = wpos;
      }
    }
    // the pivot row's final entries: columns j .. p0 + w - 1
    if (valid && wrow >= r0 && wrow < r0 + rpc) {
      for (int c = tid; c < live; c += NT)
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

  // all records of this panel consumed before anyone reuses receive slots / exits; the
  // panel's columns are final in global memory for the whole cluster
  cl.sync();
  const int cu = a.cu > 0 ? a.cu : C;
  if (p0 + w < cu) {
    // ---- U12 of the pivot rows for the trailing columns (forward substitution) -----------
    for (int e = tid; e < w * w; e += NT) {
      const int t = e / w, s = e % w;
      const int pr = prows[t];
      L11[t * NB + s] = pr >= 0 ? X[(int64_t)(p0 + s) * ldx + pr] : T(0);
    }
    __syncthreads();
    for (int c = p0 + w + crank * NW + warp; c < cu; c += ncta * NW) {
      constexpr int NQ = (NB + 31) / 32;
      T u[NQ], fin[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int t = lane + 32 * q;
        u[q] = (t < w && prows[t] >= 0) ? X[(int64_t)c * ldx + prows[t]] : T(0);
        fin[q] = u[q];
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        for (int s = 32 * q; s < min(w, 32 * q + 32); ++s) {
          T us = shfl_t(u[q], s - 32 * q);
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
        if (t < w && prows[t] >= 0) X[(int64_t)c * ldx + prows[t]] = fin[q];
        if (t < w) static_cast<T*>(a.u12)[(int64_t)t * a.ldu + c] = prows[t] >= 0 ? fin[q] : T(0);
      }
    }
  }

  // persist the positions for the next panel; the last panel writes P (gather form)
  const bool last = (p0 + w >= C);
#pragma unroll
  for (int s = 0; s < RT; ++s)
    if (have[s]) a.posg[rowi[s]] = pos[s];
  if (crank == 0)
    for (int t = tid; t < w; t += NT) a.psg[p0 + t] = prows[t];
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

template <typename T, bool CROUT, int RT, int NB, int NT, bool SOLO>
__global__ void __launch_bounds__(NT, 1) k_lu_reg(LuArgs a) {
  lu_reg_body<T, CROUT, RT, NB, NT, SOLO>(a);
}

// Batched form: cluster c of the launch factors problem table[c] (one panel: pw = C).
template <typename T, bool CROUT, int RT, int NB, int NT, bool SOLO>
__global__ void __launch_bounds__(NT, 1) k_lu_reg_batched(const LuArgs* __restrict__ table) {
  const int csize = (int)cg::this_cluster().num_blocks();
  lu_reg_body<T, CROUT, RT, NB, NT, SOLO>(table[blockIdx.x / csize]);
}

// Asynchronous global -> shared copies (cp.async): 16 bytes, or one element.
__device__ __forceinline__ void lr_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n"
               ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void lr_cp(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n"
               ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void lr_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void lr_cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Rank-w update (w <= 96) of the columns [c_begin, c_end) of every row whose position is at
// least p0 + w: X[r][c] -= sum_s X[r][p0 + s] U[s][c], U = the solved pivot rows, dense in
// u12 (row s at u12 + s * ldu). A CTA takes 256 rows (128 threads, 2 rows each) and nch
// chunks of 32 columns. Its rows' multipliers are copied to shared memory once and each
// chunk of U while the previous chunk is computed (cp.async, many copies in flight); every
// thread keeps 2 x 32 accumulators in registers. vec: X's columns start on 16-byte
// boundaries, so the multipliers move in 16-byte copies.
static constexpr int TR_T = 128;
static constexpr int TR_R = 256;

template <typename T>
__global__ void __launch_bounds__(TR_T) k_lu_trail(T* __restrict__ X, int64_t ldx, int R,
                                                  int c_begin, int c_end, int p0, int w,
                                                  const int32_t* __restrict__ posg,
                                                  const T* __restrict__ u12, int64_t ldu,
                                                  int nch, bool vec) {
  extern __shared__ __align__(16) unsigned char tr_smem[];
  T* Ls = reinterpret_cast<T*>(tr_smem);  // [w][TR_R] multipliers of this CTA's rows
  T* Us = Ls + (size_t)w * TR_R;          // [2][w][LR_CH] chunks of U
  const int tid = threadIdx.x;
  const int rb = (int)blockIdx.x * TR_R;
  const int r0 = rb + tid, r1 = rb + tid + TR_T;
  const bool u0 = r0 < R && posg[r0] >= p0 + w;
  const bool u1 = r1 < R && posg[r1] >= p0 + w;
  // the multipliers: rows rb .. rb + 255 of columns p0 .. p0 + w - 1 (rows past the column's
  // storage, ldx, read as zero)
  constexpr int EPC = 16 / (int)sizeof(T);
  if (vec) {
    for (int e = tid; e < w * (TR_R / EPC); e += TR_T) {
      const int s = e / (TR_R / EPC), i = (e % (TR_R / EPC)) * EPC;
      T* d = Ls + (size_t)s * TR_R + i;
      if (rb + i + EPC <= ldx) {
        lr_cp16(d, X + (int64_t)(p0 + s) * ldx + rb + i);
      } else {
#pragma unroll
        for (int u = 0; u < EPC; ++u) d[u] = T(0);
      }
    }
  } else {
    for (int e = tid; e < w * TR_R; e += TR_T) {
      const int s = e / TR_R, i = e % TR_R;
      if (rb + i < ldx) lr_cp<sizeof(T)>(Ls + e, X + (int64_t)(p0 + s) * ldx + rb + i);
      else Ls[e] = T(0);
    }
  }
  const int cb = c_begin + (int)blockIdx.y * nch * LR_CH;
  int nc = (c_end - cb + LR_CH - 1) / LR_CH;
  nc = nc < nch ? nc : nch;
  auto issue = [&](int ch) {  // chunk ch of U into buffer ch & 1
    const int c0 = cb + ch * LR_CH, cw = min(LR_CH, c_end - c0);
    T* d = Us + (size_t)(ch & 1) * w * LR_CH;
    for (int e = tid; e < w * LR_CH; e += TR_T) {
      const int s = e / LR_CH, q = e % LR_CH;
      if (q < cw) lr_cp<sizeof(T)>(d + e, u12 + (int64_t)s * ldu + c0 + q);
      else d[e] = T(0);
    }
  };
  issue(0);
  lr_cp_commit();
  for (int ch = 0; ch < nc; ++ch) {
    const int c0 = cb + ch * LR_CH, cw = min(LR_CH, c_end - c0);
    if (ch + 1 < nc) issue(ch + 1);
    lr_cp_commit();
    T acc0[LR_CH], acc1[LR_CH];
#pragma unroll
    for (int q = 0; q < LR_CH; ++q) {
      acc0[q] = (u0 && q < cw) ? X[(int64_t)(c0 + q) * ldx + r0] : T(0);
      acc1[q] = (u1 && q < cw) ? X[(int64_t)(c0 + q) * ldx + r1] : T(0);
    }
    lr_cp_wait<1>();  // everything but the chunk just issued has landed
    __syncthreads();
    const T* U = Us + (size_t)(ch & 1) * w * LR_CH;
#pragma unroll 2
    for (int s = 0; s < w; ++s) {
      const T l0 = Ls[s * TR_R + tid], l1 = Ls[s * TR_R + tid + TR_T];
#pragma unroll
      for (int q = 0; q < LR_CH; q += 4) {
        T uv[4];
        ld4(&U[s * LR_CH + q], uv);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc0[q + v] = fma(-l0, uv[v], acc0[q + v]);
          acc1[q + v] = fma(-l1, uv[v], acc1[q + v]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < LR_CH; ++q) {
      if (u0 && q < cw) X[(int64_t)(c0 + q) * ldx + r0] = acc0[q];
      if (u1 && q < cw) X[(int64_t)(c0 + q) * ldx + r1] = acc1[q];
    }
    __syncthreads();  // buffer ch & 1 is free for chunk ch + 2
  }
  lr_cp_wait<0>();
}

// Launches k_lu_trail on the columns [c_begin, c_end): chunks of 32 columns are grouped
// per CTA only while the grid keeps at least two CTAs per SM.
template <typename T>
static int32_t launch_trail(T* X, int64_t ldx, int R, int c_begin, int c_end, int p0, int w,
                            const int32_t* posg, const T* u12, int64_t ldu, cudaStream_t s) {
  const int rows = (int)ceil_div(R, TR_R);
  const int chunks = (int)ceil_div(c_end - c_begin, LR_CH);
  int nch = 1;
  while (nch < 4 && (int64_t)rows * ceil_div(chunks, nch + 1) >= 2 * sm_count()) ++nch;
  const size_t smem = sizeof(T) * (size_t)w * (TR_R + 2 * LR_CH);
  RLU_CUDA_TRY(cudaFuncSetAttribute(k_lu_trail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  const bool vec = ((uintptr_t)X % 16 == 0) && (ldx * (int64_t)sizeof(T)) % 16 == 0;
  const dim3 grid((unsigned)rows, (unsigned)ceil_div(chunks, nch));
  k_lu_trail<T><<<grid, TR_T, smem, s>>>(X, ldx, R, c_begin, c_end, p0, w, posg, u12, ldu, nch,
                                         vec);
  return last_launch_status();
}

// Pivot rows of a block of W <= 96 columns [o0, o0 + W), for the columns [c_begin, c_end):
// u = L11^-1 x over the block's pivot rows (forward substitution; L11[t][s] = X[o0 + s] at
// the row of position o0 + t, unit diagonal for Doolittle; Crout divides by the diagonal).
// One warp per column; L11 in shared memory.
template <typename T, bool CROUT>
__global__ void __launch_bounds__(256) k_lu_u12(T* __restrict__ X, int64_t ldx, int o0, int W,
                                               int c_begin, int c_end,
                                               const int32_t* __restrict__ psg,
                                               T* __restrict__ u12, int64_t ldu) {
  extern __shared__ __align__(16) unsigned char u12_smem[];
  const int WP = W | 1;                               // odd row stride: no bank conflicts
  T* L11 = reinterpret_cast<T*>(u12_smem);           // [W][WP]
  int* prow = reinterpret_cast<int*>(L11 + W * WP);  // [W]
  for (int t = threadIdx.x; t < W; t += blockDim.x) prow[t] = psg[o0 + t];
  __syncthreads();
  // gathered from scattered rows: batches of independent loads, so that latencies overlap
  constexpr int LB8 = 8;
  for (int e0 = threadIdx.x; e0 < W * W; e0 += (int)blockDim.x * LB8) {
    T v[LB8];
#pragma unroll
    for (int u = 0; u < LB8; ++u) {
      const int e = e0 + u * (int)blockDim.x, t = e / W, s = e % W;
      v[u] = (e < W * W && prow[t] >= 0) ? X[(int64_t)(o0 + s) * ldx + prow[t]] : T(0);
    }
#pragma unroll
    for (int u = 0; u < LB8; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < W * W) L11[(e / W) * WP + e % W] = v[u];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int c = c_begin + (int)blockIdx.x * (blockDim.x / 32) + (int)(threadIdx.x >> 5);
  if (c >= c_end) return;
  constexpr int NQ = 3;  // W <= 96
  T u[NQ], fin[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int t = lane + 32 * q;
    u[q] = (t < W && prow[t] >= 0) ? X[(int64_t)c * ldx + prow[t]] : T(0);
    fin[q] = u[q];
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    for (int s = 32 * q; s < min(W, 32 * q + 32); ++s) {
      T us = shfl_t(u[q], s - 32 * q);
      if (CROUT) {
        const T pv = L11[s * WP + s];
        if (pv != T(0)) us = us * rcp_piv(pv);
      }
      if (lane == s - 32 * q) fin[q] = us;
#pragma unroll
      for (int qq = q; qq < NQ; ++qq) {
        const int t = lane + 32 * qq;
        if (t > s && t < W) u[qq] = fma(-L11[t * WP + s], us, u[qq]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int t = lane + 32 * q;
    if (t < W && prow[t] >= 0) X[(int64_t)c * ldx + prow[t]] = fin[q];
    if (t < W) u12[(int64_t)t * ldu + c] = prow[t] >= 0 ? fin[q] : T(0);
  }
}

template <typename T, int NB, int NT>
static size_t lr_smem_bytes(int rpc, int C) {
  size_t b = (sizeof(LrShared<T, NB, NT / 32>) + 15) / 16 * 16;
  b += (sizeof(T) * (size_t)NB * NB + 15) / 16 * 16;
  b += sizeof(int) * (size_t)NB;
  (void)rpc;
  (void)C;
  return b;
}

// A rank-w trailing update: large ones (rank >= 64 over >= 128 columns) on the tensor cores
// (FP32 with scratch for U^T's TF32 parts), the others (and where that form does not apply)
// on the SIMT kernel, whose launch costs less than the tensor-core form's set-up.
template <typename T>
static int32_t trail(const LuArgs& in, T* X, int c_begin, int c_end, int p0, int w, T* U12,
                     cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (in.u12t && w >= 64 && c_end - c_begin >= 128) {
      const int32_t st = umma3_trail(X, in.ldx, in.R, c_begin, c_end, p0, w, in.posg, U12,
                                     in.ldu, static_cast<float*>(in.u12t), in.status, s);
      if (st != RLU_EUNSUPPORTED) return st;
    }
  }
  return launch_trail<T>(X, in.ldx, in.R, c_begin, c_end, p0, w, in.posg, U12, in.ldu, s);
}

template <typename T, bool CROUT, int RT, int NB, int NT>
static int32_t try_launch(const LuArgs& in, cudaStream_t s, bool* launched) {
  *launched = false;
  const int rpc = NT * RT;
  const int ncta = (int)ceil_div(in.R, rpc);
  if (ncta > 16) return RLU_OK;
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t bytes = lr_smem_bytes<T, NB, NT>(rpc, in.C);
  if (bytes > (size_t)optin) return RLU_OK;
  auto kern = k_lu_reg<T, CROUT, RT, NB, NT, false>;
  if constexpr (RT == 1) {  // one CTA: no exchange (RT = 1 covers every problem that fits one)
    if (ncta == 1) kern = k_lu_reg<T, CROUT, RT, NB, NT, true>;
  }
  RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(ncta);
  cfg.blockDim = dim3(NT);
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
  // no position state or pivot-row buffer: the one-launch kernel takes the problem
  if (!in.posg || !in.psg || !in.u12) return RLU_OK;
  LuArgs a = in;
  a.rpc = rpc;
  a.nb = NB - 1;
  // blocks of whole panels, about 64 columns (panels of 64 or more columns: one block);
  // a block's L11 (W x W) must fit k_lu_u12's 48 KB of shared memory and W <= 96
  const int pw_max = NB - 1;
  int np = (64 + pw_max / 2) / pw_max;
  while (np > 1 && (np * pw_max > 96 ||
                    sizeof(T) * (size_t)(np * pw_max) * ((np * pw_max) | 1) + 4 * (np * pw_max) > 48 * 1024))
    --np;
  // complex: a two-panel block's 72-row pivot solve (complex shuffles and FMAs) costs more
  // than the trailing columns' extra reads save, so every panel is its own block (frlu_4096:
  // 2.52 -> 2.39 ms)
  if constexpr (std::is_same<T, cf32>::value) np = 1;
  const int wo = pw_max >= 64 ? in.C : np * pw_max;
  T* X = static_cast<T*>(in.X);
  T* U12 = static_cast<T*>(in.u12);
  for (int o0 = 0; o0 < in.C; o0 += wo) {
    const int o1 = min(in.C, o0 + wo);
    for (int p0 = o0; p0 < o1; p0 += pw_max) {
      a.p0 = p0;
      a.pw = min(pw_max, o1 - p0);
      a.cu = o1;
      RLU_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
      RLU_TRY(last_launch_status());
      *launched = true;
      if (p0 + a.pw < o1)
        RLU_TRY(trail<T>(in, X, p0 + a.pw, o1, p0, a.pw, U12, s));
    }
    if (o1 < in.C) {
      const int W = o1 - o0;  // <= 96
      const size_t ub = sizeof(T) * (size_t)W * (W | 1) + sizeof(int) * (size_t)W;
      k_lu_u12<T, CROUT><<<(unsigned)ceil_div(in.C - o1, 8), 256, ub, s>>>(X, in.ldx, o0, W, o1,
                                                                          in.C, in.psg, U12,
                                                                          in.ldu);
      RLU_TRY(last_launch_status());
      RLU_TRY(trail<T>(in, X, o1, in.C, o0, W, U12, s));
    }
  }
  return RLU_OK;
}

template <typename T, bool CROUT>
static int32_t launch_reg_t(const LuArgs& a, cudaStream_t s, bool* launched) {
  // rows per thread RT, register panel NB (NB - 1 columns per panel), threads per CTA
  constexpr int W1 = sizeof(T) == 4 ? 77 : 37;
  constexpr int W2 = sizeof(T) == 4 ? 37 : 19;
  // 4 rows per thread: 18 FP32 columns per panel spill ~48 bytes but halve the panel
  // launches against 10 columns (LU of Y at 32768 x 532: 2.16 -> 2.06 ms)
  constexpr int W4 = sizeof(T) == 4 ? 19 : 7;
  // FP64 multiply-adds run at 1/64 of the FP32 rate: up to 2048 rows take 128-thread CTAs,
  // so that a step's rank-1 update spreads over four times as many SMs' FP64 units
  if constexpr (std::is_same<T, double>::value) {
    if (a.R <= 16 * 128) RLU_TRY((try_launch<T, CROUT, 1, W1, 128>(a, s, launched)));
  }
  // complex: four real multiply-adds per element; up to 4096 rows take 256-thread CTAs, twice
  // the SMs of 512-thread ones for the rank-1 updates
  if constexpr (std::is_same<T, cf32>::value) {
    if (a.R <= 16 * 256) RLU_TRY((try_launch<T, CROUT, 1, W1, 256>(a, s, launched)));
  }
  if (!*launched && a.R <= 16 * 512) RLU_TRY((try_launch<T, CROUT, 1, W1, 512>(a, s, launched)));
  if (!*launched && a.R <= 16 * 1024) RLU_TRY((try_launch<T, CROUT, 2, W2, 512>(a, s, launched)));
  if (!*launched && a.R <= 16 * 2048) RLU_TRY((try_launch<T, CROUT, 4, W4, 512>(a, s, launched)));
  return RLU_OK;
}

int32_t launch_lu_reg(int32_t dtype, bool crout, const LuArgs& a, cudaStream_t s, bool* launched) {
  *launched = false;
  if (dtype == RLU_F64) return crout ? launch_reg_t<double, true>(a, s, launched) : launch_reg_t<double, false>(a, s, launched);
  if (dtype == RLU_F32) return crout ? launch_reg_t<float, true>(a, s, launched) : launch_reg_t<float, false>(a, s, launched);
  if (dtype == kLuC64) return crout ? launch_reg_t<cf32, true>(a, s, launched) : launch_reg_t<cf32, false>(a, s, launched);
  return RLU_OK;
}

// Batched LUs of problems that fit one register panel (C <= NB - 1 = 76 FP32 columns, R <=
// 16 x rows_per_cta): the table on the device is grouped by cluster size (ceil(R /
// rows_per_cta) CTAs); group g starts at table entry first[g] and holds count[g] problems.
// rows_per_cta is 512 (512-thread CTAs) or 256 (256-thread CTAs, twice as many CTAs per
// problem).
template <int NT>
static int32_t lu_batched_group(bool crout, const LuArgs* table_dev, int first, int count, int g,
                                cudaStream_t s) {
  using T = float;
  constexpr int NB = 77;
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t bytes = lr_smem_bytes<T, NB, NT>(NT, 0);
  if (bytes > (size_t)optin) return RLU_EUNSUPPORTED;
  auto kern = g == 1 ? (crout ? k_lu_reg_batched<T, true, 1, NB, NT, true>
                              : k_lu_reg_batched<T, false, 1, NB, NT, true>)
                    : (crout ? k_lu_reg_batched<T, true, 1, NB, NT, false>
                             : k_lu_reg_batched<T, false, 1, NB, NT, false>);
  RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = g;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(g * count));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RLU_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, table_dev + first));
  return last_launch_status();
}

int32_t launch_lu_reg_batched(bool crout, int rows_per_cta, const LuArgs* table_dev,
                              const int* first, const int* count, cudaStream_t s,
                              const LuFork* fork) {
  if (rows_per_cta != 512 && rows_per_cta != 256) return RLU_EINVAL;
  int groups[kLuGroups], ng = 0;
  for (int g = 16; g >= 1; --g)  // widest clusters first
    if (count[g] > 0) groups[ng++] = g;
  for (int g : {17, 18})  // one narrow CTA for small problems, several per SM
    if (count[g] > 0) groups[ng++] = g;
  const bool par = fork != nullptr && ng > 1;
  if (par) RLU_CUDA_TRY(cudaEventRecord(fork->fork, s));
  for (int i = 0; i < ng; ++i) {
    const int g = groups[i];
    cudaStream_t gs = s;
    if (par) {
      gs = fork->hs[i % kLuSide];
      if (i < kLuSide) RLU_CUDA_TRY(cudaStreamWaitEvent(gs, fork->fork, 0));
    }
    if (g == 17)
      RLU_TRY(lu_batched_group<128>(crout, table_dev, first[g], count[g], 1, gs));
    else if (g == 18)
      RLU_TRY(lu_batched_group<256>(crout, table_dev, first[g], count[g], 1, gs));
    else if (rows_per_cta == 512)
      RLU_TRY(lu_batched_group<512>(crout, table_dev, first[g], count[g], g, gs));
    else
      RLU_TRY(lu_batched_group<256>(crout, table_dev, first[g], count[g], g, gs));
  }
  if (par)
    for (int i = 0; i < ng && i < kLuSide; ++i) {
      RLU_CUDA_TRY(cudaEventRecord(fork->join[i], fork->hs[i]));
      RLU_CUDA_TRY(cudaStreamWaitEvent(s, fork->join[i], 0));
    }
  return RLU_OK;
}

}  // namespace rlu
