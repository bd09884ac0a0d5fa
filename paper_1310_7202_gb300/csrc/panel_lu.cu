// Pivoted LU of a tall-skinny column-major matrix X (R x C, R >= C) on one thread-block
// cluster: steps 3 and 6 of Algorithm 1.
//
//  * Step 3 (LU of Y with partial pivoting, the remark after Algorithm 1): X = Y (m x l),
//    Doolittle form: multipliers X[r][j]/pivot stored in column j, the pivot row unscaled.
//  * Step 6 (LU of B with column pivoting, B Q = L_b U_b): X = B^T (n x k). Pivoting on the
//    largest entry of row j of B is pivoting on column j of B^T; keeping the unit diagonal
//    on L_b means the pivot ROW of X is divided by the pivot ("Crout" form) while column j
//    keeps the unscaled values, which are the entries U_b[j][.] of B's factor.
//
// Rows never move ("swap-free"). Each row carries its current position pos[r]; the pivot of
// step j is the candidate with the largest |value| and, among equal magnitudes, the smallest
// current position, which is exactly the row LAPACK getf2 would pick after its physical
// swaps. Swapping positions j and pos[b] is a bookkeeping update of two integers. perm[p]
// (row at final position p) is P in gather form.
//
// The cluster (1..16 CTAs) splits the rows into contiguous blocks; a panel of nb columns of
// the CTA's rows lives in its shared memory. Per step: local argmax (warp shuffles), one
// cluster barrier, every CTA reduces the cluster's candidates from distributed shared memory
// and copies the pivot row from its owner, then updates its own rows. After a panel:
// (i) the pivot rows' trailing entries (U12) by forward substitution with the panel's
// L11 (one warp per trailing column), (ii) the rank-nb update of every non-pivot row's
// trailing columns in global memory (L2-resident).
#include <cooperative_groups.h>

#include "common.cuh"
#include "panel_lu.cuh"

namespace cg = cooperative_groups;

namespace rlu {

static constexpr int LU_NT = 512;
static constexpr int LU_NW = LU_NT / 32;
static constexpr int LU_CH = 32;      // trailing-update column chunk
static constexpr int LU_NBMAX = 128;  // widest panel (U12 forward substitution: 4 per lane)

// Dynamic shared memory: panel [nb][rpc], L11 [nb][nb] and U12 chunk [nb][LU_CH] (only when
// the columns need more than one panel), pivot rows [2][nb], positions [rpc], map [C].
template <typename T>
static size_t lu_smem_bytes(int nb, int rpc, int C, bool multi) {
  const size_t extra = multi ? (size_t)nb * nb + (size_t)nb * LU_CH : 0;
  return sizeof(T) * ((size_t)nb * rpc + extra + 2 * (size_t)nb) +
         sizeof(int) * ((size_t)rpc + (size_t)C);
}

template <typename T, bool CROUT>
__global__ void __launch_bounds__(LU_NT, 1) k_cluster_lu(LuArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int ncta = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rpc = a.rpc, nb = a.nb, C = a.C;
  const int r0 = crank * rpc;
  const int nr = max(0, min(rpc, a.R - r0));
  const int64_t ldx = a.ldx;
  T* __restrict__ X = static_cast<T*>(a.X);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const bool multi = nb < C;
  T* Xs = reinterpret_cast<T*>(smem_raw);  // [nb][rpc]
  T* L11 = Xs + (size_t)nb * rpc;          // [nb][nb]: (t, s) at t*nb + s (multi only)
  T* U12 = L11 + (multi ? (size_t)nb * nb : 0);        // [nb][LU_CH] (multi only)
  T* prow = U12 + (multi ? (size_t)nb * LU_CH : 0);    // [2][nb]
  int* posl = reinterpret_cast<int*>(prow + 2 * nb);  // [rpc]
  int* psmall = posl + rpc;                           // [C]: row at position p < C

  __shared__ T s_part_mag[2];
  __shared__ int s_part_pos[2], s_part_row[2];
  __shared__ T s_wmag[LU_NW];
  __shared__ int s_wpos[LU_NW], s_wrow[LU_NW];
  __shared__ T s_win_mag;
  __shared__ int s_win_pos, s_win_row;
  __shared__ int s_nonfinite;

  for (int t = tid; t < nr; t += LU_NT) posl[t] = r0 + t;
  for (int p = tid; p < C; p += LU_NT) psmall[p] = p;
  if (tid == 0) s_nonfinite = 0;
  int first_zero = -1;
  __syncthreads();

  // deferred write-back of a scaled pivot row (Crout form)
  int prev_owner = -1, prev_lr = 0, prev_par = 0;
  bool prev_nz = false;

  for (int p0 = 0; p0 < C; p0 += nb) {
    const int w = min(nb, C - p0);
    for (int jj = 0; jj < w; ++jj) {
      const T* src = X + (int64_t)(p0 + jj) * ldx + r0;
      for (int t = tid; t < nr; t += LU_NT) Xs[(size_t)jj * rpc + t] = src[t];
    }
    prev_owner = -1;
    __syncthreads();

    for (int jj = 0; jj < w; ++jj) {
      const int j = p0 + jj;
      const int par = j & 1;
      // ---- local candidate -------------------------------------------------------------
      T bm = T(-1);
      int bp = INT_MAX, br = -1;
      bool nf = false;
      for (int t = tid; t < nr; t += LU_NT) {
        const int ps = posl[t];
        if (ps >= j) {
          const T v = Xs[(size_t)jj * rpc + t];
          nf |= !is_finite_val(v);
          const T mg = fabs(v);
          if (cand_better(mg, ps, bm, bp)) {
            bm = mg;
            bp = ps;
            br = r0 + t;
          }
        }
      }
      if (nf) s_nonfinite = 1;
      warp_argmax(bm, bp, br);
      if (lane == 0) {
        s_wmag[warp] = bm;
        s_wpos[warp] = bp;
        s_wrow[warp] = br;
      }
      __syncthreads();
      if (warp == 0) {
        bm = lane < LU_NW ? s_wmag[lane] : T(-1);
        bp = lane < LU_NW ? s_wpos[lane] : INT_MAX;
        br = lane < LU_NW ? s_wrow[lane] : -1;
        warp_argmax(bm, bp, br);
        if (lane == 0) {
          s_part_mag[par] = bm;
          s_part_pos[par] = bp;
          s_part_row[par] = br;
        }
      }
      cl.sync();
      // ---- deferred write-back of the previous step's scaled pivot row ----------------
      if (CROUT && prev_owner == crank && prev_nz) {
        for (int c = jj + tid; c < w; c += LU_NT)
          Xs[(size_t)c * rpc + prev_lr] = prow[prev_par * nb + c];
      }
      // ---- cluster-wide winner -------------------------------------------------------
      if (warp == 0) {
        bm = T(-1);
        bp = INT_MAX;
        br = -1;
        if (lane < ncta) {
          bm = *cl.map_shared_rank(&s_part_mag[par], lane);
          bp = *cl.map_shared_rank(&s_part_pos[par], lane);
          br = *cl.map_shared_rank(&s_part_row[par], lane);
        }
        warp_argmax(bm, bp, br);
        if (lane == 0) {
          s_win_mag = bm;
          s_win_pos = bp;
          s_win_row = br;
        }
      }
      __syncthreads();
      const int wrow = s_win_row, wpos = s_win_pos;
      const bool valid = wrow >= 0;
      const bool nz = valid && s_win_mag != T(0);
      const int owner = valid ? wrow / rpc : 0;
      const int lr = valid ? wrow - owner * rpc : 0;
      // ---- pivot row: columns jj..w-1 from the owner's shared memory -----------------
      if (valid) {
        const T* rX = cl.map_shared_rank(Xs, owner);
        for (int c = jj + tid; c < w; c += LU_NT) prow[par * nb + c] = rX[(size_t)c * rpc + lr];
      }
      const int a_row = psmall[j];
      __syncthreads();
      const T piv = prow[par * nb + jj];
      if (CROUT && nz) {
        for (int c = jj + 1 + tid; c < w; c += LU_NT) prow[par * nb + c] = prow[par * nb + c] / piv;
      }
      // ---- position bookkeeping ------------------------------------------------------
      if (tid == 0) {
        if (valid && wrow != a_row) {
          psmall[j] = wrow;
          if (wpos < C) psmall[wpos] = a_row;
          if (a_row >= r0 && a_row < r0 + nr) posl[a_row - r0] = wpos;
          if (wrow >= r0 && wrow < r0 + nr) posl[wrow - r0] = j;
        }
        if (!nz && first_zero < 0) first_zero = j;
      }
      __syncthreads();
      // ---- eliminate below the pivot (own rows) ---------------------------------------
      if (nz) {
        const T* pr = prow + par * nb;
        for (int t = tid; t < nr; t += LU_NT) {
          if (posl[t] > j) {
            const T x = Xs[(size_t)jj * rpc + t];
            const T mlt = CROUT ? x : x / piv;
            if (!CROUT) Xs[(size_t)jj * rpc + t] = mlt;
            for (int c = jj + 1; c < w; ++c)
              Xs[(size_t)c * rpc + t] = fma(-mlt, pr[c], Xs[(size_t)c * rpc + t]);
          }
        }
      }
      prev_owner = valid ? owner : -1;
      prev_lr = lr;
      prev_nz = nz;
      prev_par = par;
    }
    cl.sync();  // every pivot-row read of this panel is done

    for (int jj = 0; jj < w; ++jj) {
      T* dst = X + (int64_t)(p0 + jj) * ldx + r0;
      for (int t = tid; t < nr; t += LU_NT) dst[t] = Xs[(size_t)jj * rpc + t];
    }
    if (p0 + w >= C) break;
    cl.sync();  // the panel in global memory is visible to the cluster

    // ---- (i) U12 = L11^{-1} X(pivot rows, trailing) (Crout: then scaled by the pivot) ---
    for (int e = tid; e < w * w; e += LU_NT) {
      const int t = e / w, s = e % w;
      L11[t * nb + s] = X[(int64_t)(p0 + s) * ldx + psmall[p0 + t]];
    }
    __syncthreads();
    for (int c = p0 + w + crank * LU_NW + warp; c < C; c += ncta * LU_NW) {
      T u[LU_NBMAX / 32], fin[LU_NBMAX / 32];
#pragma unroll
      for (int q = 0; q < LU_NBMAX / 32; ++q) {
        const int t = lane + 32 * q;
        u[q] = t < w ? X[(int64_t)c * ldx + psmall[p0 + t]] : T(0);
        fin[q] = u[q];
      }
#pragma unroll
      for (int q = 0; q < LU_NBMAX / 32; ++q) {
        for (int s = 32 * q; s < min(w, 32 * q + 32); ++s) {
          T us = __shfl_sync(0xffffffffu, u[q], s - 32 * q);
          if (CROUT) {
            const T pv = L11[s * nb + s];
            if (pv != T(0)) us = us / pv;
          }
          if (lane == s - 32 * q) fin[q] = us;
#pragma unroll
          for (int qq = q; qq < LU_NBMAX / 32; ++qq) {
            const int t = lane + 32 * qq;
            if (t > s && t < w) u[qq] = fma(-L11[t * nb + s], us, u[qq]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < LU_NBMAX / 32; ++q) {
        const int t = lane + 32 * q;
        if (t < w) X[(int64_t)c * ldx + psmall[p0 + t]] = fin[q];
      }
    }
    cl.sync();  // U12 visible

    // ---- (ii) trailing update of this CTA's non-pivot rows -----------------------------
    for (int cc = p0 + w; cc < C; cc += LU_CH) {
      const int cw = min(LU_CH, C - cc);
      for (int e = tid; e < w * LU_CH; e += LU_NT) {
        const int s = e / LU_CH, q = e % LU_CH;
        U12[s * LU_CH + q] = q < cw ? X[(int64_t)(cc + q) * ldx + psmall[p0 + s]] : T(0);
      }
      __syncthreads();
      for (int t = tid; t < nr; t += LU_NT) {
        if (posl[t] < p0 + w) continue;
        T acc[LU_CH];
#pragma unroll
        for (int q = 0; q < LU_CH; ++q)
          acc[q] = q < cw ? X[(int64_t)(cc + q) * ldx + r0 + t] : T(0);
        for (int s = 0; s < w; ++s) {
          const T lv = Xs[(size_t)s * rpc + t];
#pragma unroll
          for (int q = 0; q < LU_CH; ++q) acc[q] = fma(-lv, U12[s * LU_CH + q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < LU_CH; ++q)
          if (q < cw) X[(int64_t)(cc + q) * ldx + r0 + t] = acc[q];
      }
      __syncthreads();
    }
    cl.sync();
  }

  for (int t = tid; t < nr; t += LU_NT) a.perm[posl[t]] = r0 + t;
  if (tid == 0) {
    if (crank == 0 && a.zero_step && first_zero >= 0) atomicCAS(a.zero_step, -1, first_zero);
    if (s_nonfinite && a.nonfinite) atomicOr(a.nonfinite, 1);
  }
  cl.sync();  // keep shared memory alive until every remote read has finished
}

// ---------------------------------------------------------------------------------------
template <typename T, bool CROUT>
static int32_t launch_lu_t(const LuArgs& in, cudaStream_t s) {
  static bool attr_done[64] = {false};
  int dev = 0;
  RLU_CUDA_TRY(cudaGetDevice(&dev));
  int smem_optin = 0;
  RLU_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t budget = (size_t)smem_optin - 2048;  // static shared memory and slack
  auto kern = k_cluster_lu<T, CROUT>;
  if (dev < 64 && !attr_done[dev]) {
    RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)budget));
    RLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    attr_done[dev] = true;
  }
  const int R = in.R, C = in.C;
  auto launchable = [&](int cand, size_t bytes) -> bool {
    if (cand <= 8) return true;  // portable cluster sizes
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cand;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cand);
    cfg.blockDim = dim3(LU_NT);
    cfg.dynamicSmemBytes = bytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return nclusters >= 1;
  };
  int ncta = 0, nb = 0, rpc = 0;
  // the smallest cluster that holds all C columns in one panel ...
  const int sizes[5] = {1, 2, 4, 8, 16};
  for (int i = 0; i < 5 && ncta == 0; ++i) {
    const int r = (int)round_up(ceil_div(R, sizes[i]), 4);
    const size_t bytes = lu_smem_bytes<T>(C, r, C, false);
    if (bytes <= budget && launchable(sizes[i], bytes)) {
      ncta = sizes[i];
      rpc = r;
      nb = C;
    }
  }
  // ... else the largest launchable cluster with panels of nb <= LU_NBMAX columns
  const int order[2] = {16, 8};
  for (int i = 0; i < 2 && ncta == 0; ++i) {
    const int cand = order[i];
    const int r = (int)round_up(ceil_div(R, cand), 4);
    int w = C - 1 < LU_NBMAX ? C - 1 : LU_NBMAX;
    while (w > 0 && lu_smem_bytes<T>(w, r, C, true) > budget) --w;
    if (w < 1 || !launchable(cand, lu_smem_bytes<T>(w, r, C, true))) continue;
    ncta = cand;
    rpc = r;
    nb = w;
  }
  if (ncta == 0) return RLU_EUNSUPPORTED;
  LuArgs a = in;
  a.rpc = rpc;
  a.nb = nb;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(ncta);
  cfg.blockDim = dim3(LU_NT);
  cfg.dynamicSmemBytes = lu_smem_bytes<T>(nb, rpc, C, nb < C);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RLU_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
  return last_launch_status();
}

int32_t launch_cluster_lu(int32_t dtype, bool crout, const LuArgs& a, cudaStream_t s) {
  if (a.R < a.C || a.C < 1) return RLU_EINVAL;
  bool launched = false;
  RLU_TRY(launch_lu_reg(dtype, crout, a, s, &launched));
  if (launched) return RLU_OK;
  if (dtype == RLU_F64) return crout ? launch_lu_t<double, true>(a, s) : launch_lu_t<double, false>(a, s);
  if (dtype == RLU_F32) return crout ? launch_lu_t<float, true>(a, s) : launch_lu_t<float, false>(a, s);
  return RLU_EUNSUPPORTED;
}

}  // namespace rlu
