// H_eff . theta with a U(1) symmetry (particle-number conservation), every
// sector block of each GEMM stage in one grouped persistent launch.
//
// With a conserved charge every bond index carries a charge and the tensors
// are block sparse: theta[a,s1,s2,c] != 0 only if q(a) + s1 + s2 = q(c) (a
// local state s carries charge s), L[a2,w,a] only if q(a2) = q(a) + q_w,
// R[c2,w,c] only if q(c2) = q(c) + q_w. The product of Sec. 3.4
// (Fig. LanczosMPS) then splits into blocks:
//   stage 1, one problem per ket sector i of a: T1_i[(w,a2), (s1,s2,c)] =
//            L[(w,a2), a in i] . theta_i[a, (s1,s2,c)]
//   stages 2+3 (fused): T3_j[(t1,t2,a2), (w2,c)] =
//            sum_{w,s1} Wc[t1,t2,w2][w,s1,s2] T1_{i(a2,w)}[(w,a2), (s1,s2,c)],
//            Wc = sum_w1 W1[w,t1,s1,w1] W2[w1,t2,s2,w2], s2 fixed by the charges
//   stage 4, one problem per output sector j of c2: Y_j[(t1,t2,a2), c2] =
//            T3_j[(t1,t2,a2), (w2,c)] . R[c2 in j, (w2,c)]
// and the rows of Y_j are scattered into y. Stages 1 and 4 are one grouped
// tcgen05 launch each (split precision, as in the dense path).
//
// Packed format of theta, y, L and R: the entries allowed by the charge rule,
// in C order of the dense tensor (numpy: dense[mask]). Sectors are listed in
// bond-index order, so each allowed run along the last index is one sector.
#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include <atomic>

#include "common.cuh"
#include "ieee.cuh"

struct osmps_u1_heff {
  osmps_ctx* ctx = nullptr;
  uint64_t uid = 0;  // unique per plan in the process (keys recorded Lanczos graphs)
  int64_t nl = 0, nr = 0, d1 = 0, d2 = 0, wl = 0, wm = 0, wr = 0;
  std::vector<int64_t> ql, chil, qr, chir, qwl, qwr;
  int64_t qmin = 0, nq = 0;
  int64_t n_theta = 0, n_L = 0, n_R = 0;
  double flops1 = 0.0, flops4 = 0.0;
  // stage 1 / stage 4 problems (nkb filled per operand type) and their K padding
  std::vector<osmps::GroupProblem> p1, p4;
  std::vector<int64_t> kp1, kp4;
  int64_t tiles1 = 0, rowsA1 = 0, rowsB1 = 0, Kpl1 = 64, n_T1 = 0;
  int64_t tiles4 = 0, rowsA4 = 0, rowsB4 = 0, Kpl4 = 64, n_Y = 0;
  int64_t n_A4 = 0;  // stage-4 A entries the W-step writes (sum over rows of the row's K)
  int kind_loaded = -1;    // operand type of the problem table on the device
  int prepared_kind = -1;  // operand type of the prepared L, R operands (-1: none)
  // device memory
  int64_t* d_tab = nullptr;
  osmps::GroupProblem* d_prob = nullptr;
  // tile width each grouped stage's table is built for, and whether it is
  // settled (measured or taken from the context's tuning table)
  int bn1 = 256, bn4 = 256;
  bool settled1 = false, settled4 = false;
  uint8_t* d_buf = nullptr;
  // offsets (int64 elements) of the tables inside d_tab
  int64_t t_lsec = 0, t_ql = 0, t_qr = 0, t_qwl = 0, t_rowlen = 0, t_t1off = 0, t_rs1 = 0, t_cs = 0,
          t_a1src = 0, t_a1len = 0, t_b1base = 0, t_b1stride = 0, t_b1len = 0, t_a4row = 0,
          t_a4col = 0, t_a4kp = 0, t_b4src = 0, t_b4len = 0, t_ysrc = 0, t_ydst = 0, t_ylen = 0,
          t_seg = 0, t_pseg = 0, t_rowbase = 0, t_c0tab = 0;
  // byte offsets of the buffers inside d_buf
  size_t o_A1 = 0, o_B1 = 0, o_T1 = 0, o_A4 = 0, o_B4 = 0, o_Wc = 0, o_Y = 0;
};

namespace osmps {
namespace {

int64_t find_sector(const std::vector<int64_t>& q, int64_t charge) {
  for (size_t i = 0; i < q.size(); ++i)
    if (q[i] == charge) return (int64_t)i;
  return -1;
}

int ew_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), 65536)); }

template <int KIND>
__device__ __forceinline__ void store_split_f(void* dst, int64_t off_hi, int64_t Kpl, float x) {
  if (KIND == TC_BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    reinterpret_cast<__nv_bfloat16*>(dst)[off_hi] = h;
    reinterpret_cast<__nv_bfloat16*>(dst)[off_hi + Kpl] = l;
  } else {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float r = x - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
    reinterpret_cast<uint32_t*>(dst)[off_hi] = h;
    reinterpret_cast<uint32_t*>(dst)[off_hi + Kpl] = l;
  }
}

// Split of a float64 value: hi = round(x), lo = round(x - hi) in the operand
// type. The roundings and the widening of hi use the integer fields
// (ieee.cuh); only the exact subtraction x - hi runs on GB300's narrow
// float64 pipe. Bit for bit the split of the hardware conversions.
template <int KIND>
__device__ __forceinline__ void store_split_d(void* dst, int64_t off_hi, int64_t Kpl, double x) {
  if (KIND == TC_BF16) {
    const __nv_bfloat16 h = f64_to_bf16_rn(x);
    const __nv_bfloat16 l = f64_to_bf16_rn(x - f32_to_f64(__bfloat162float(h)));
    reinterpret_cast<__nv_bfloat16*>(dst)[off_hi] = h;
    reinterpret_cast<__nv_bfloat16*>(dst)[off_hi + Kpl] = l;
  } else {
    uint32_t h, l;
    const float xf = f64_to_f32_rn(x);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(xf));
    const float r = f64_to_f32_rn(x - f32_to_f64(__uint_as_float(h)));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
    reinterpret_cast<uint32_t*>(dst)[off_hi] = h;
    reinterpret_cast<uint32_t*>(dst)[off_hi + Kpl] = l;
  }
}

// Operand row r = src[row_src[r] + k] for k < row_len[r], zero up to Kpl.
template <int KIND>
__global__ void k_row_gather_split(const double* __restrict__ src, const int64_t* __restrict__ row_src,
                                   const int64_t* __restrict__ row_len, int64_t rows, int64_t Kpl,
                                   void* __restrict__ dst) {
  const int64_t total = rows * Kpl;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kpl, k = e - r * Kpl;
    const double x = k < row_len[r] ? src[row_src[r] + k] : 0.0;
    store_split_d<KIND>(dst, r * 2 * Kpl + k, Kpl, x);
  }
}

// theta^T blocks: operand row r, column k = theta[base[r] + k * stride[r]] for
// k < len[r], zero up to Kpl; 32 x 32 tiles through shared memory (reads
// along r, which is contiguous in theta, writes along k).
template <int KIND>
__global__ void k_theta_split(const double* __restrict__ th, const int64_t* __restrict__ base,
                              const int64_t* __restrict__ stride, const int64_t* __restrict__ len,
                              int64_t rows, int64_t Kpl, void* __restrict__ dst) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + tx, k = k0 + j;
    double x = 0.0;
    if (r < rows && k < len[r]) x = th[base[r] + k * stride[r]];
    tile[j][tx] = x;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + j, k = k0 + tx;
    if (r < rows && k < Kpl) store_split_d<KIND>(dst, r * 2 * Kpl + k, Kpl, tile[tx][j]);
  }
}

// Wc[((t1 d2 + t2) wr + w2) * nin + (w d1 + s1) d2 + s2] = sum_w1 W1[w,t1,s1,w1] W2[w1,t2,s2,w2]
__global__ void k_wcomb(const double* __restrict__ W1, const double* __restrict__ W2, int d1,
                        int d2, int wl, int wm, int wr, float* __restrict__ Wc) {
  const int nin = wl * d1 * d2, nout = d1 * d2 * wr;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nin * nout; e += gridDim.x * blockDim.x) {
    const int o = e / nin, i = e - o * nin;
    const int w2 = o % wr, t12 = o / wr, t2 = t12 % d2, t1 = t12 / d2;
    const int s2 = i % d2, ws1 = i / d2, s1 = ws1 % d1, w = ws1 / d1;
    double a = 0.0;
    for (int w1 = 0; w1 < wm; ++w1)
      a += W1[((int64_t)(w * d1 + t1) * d1 + s1) * wm + w1] *
           W2[((int64_t)(w1 * d2 + t2) * d2 + s2) * wr + w2];
    Wc[e] = (float)a;
  }
}

struct WstepArgs {
  const float* T1;
  const float* Wc;
  const int64_t* lsec;    // left sector index by (charge - qmin), or -1
  const int64_t* ql;      // left sector charges
  const int64_t* qr;      // right sector charges
  const int64_t* qwl;     // charge of each left MPO channel
  const int64_t* rowlen;  // per left sector: T1 row length (= theta row length)
  const int64_t* t1off;   // per left sector: T1 block offset (elements)
  const int64_t* rs1;     // [i wl + w]: first T1 row of channel w in block i, or -1
  const int64_t* cs;      // [(i d1 + s1) d2 + s2]: first column of (s1, s2) in block i, or -1
  const int64_t* a4row;   // per T3 row: {problem, t1 d2 + t2, sector of a2, a2 within it}
  const int64_t* a4col;   // per T3 column (global): {w2, sector of c, c within it}
  const int64_t* a4kp;    // per T3 row: {column base of its problem, K, Kp}
  const int64_t* seg;     // column runs of one (w2, sector of c): {w2, sector, first k, length}
  const int64_t* pseg;    // per stage-4 problem (output sector j): {first run, run count}
  const int64_t* rowbase; // [r wl + w]: T1 offset of T3 row r's channel-w row, or -1
  const int64_t* c0tab;   // [ia2 nin + (w d1 + s1) d2 + s2]: first T1 column of (s1, s2)
                          // in the ket sector q(a2) - q_w, or -1
  int64_t rows, Kpl, qmin, nq;
  int d1, d2, wl, wr;
};

// T3 written as the split operand of stage 4: one thread per (row, k < Kp of
// its problem); columns K..Kp are the zero padding.
template <int KIND>
__global__ void k_u1_wsteps(WstepArgs a, void* __restrict__ dst) {
  const int64_t r = blockIdx.y;
  if (r >= a.rows) return;
  const int64_t t12 = a.a4row[4 * r + 1], ia2 = a.a4row[4 * r + 2], a2 = a.a4row[4 * r + 3];
  const int64_t colbase = a.a4kp[3 * r], K = a.a4kp[3 * r + 1], Kp = a.a4kp[3 * r + 2];
  const int64_t qa2 = a.ql[ia2];
  const int nin = a.wl * a.d1 * a.d2;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < Kp;
       k += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.0f;
    if (k < K) {
      const int64_t* col = a.a4col + 3 * (colbase + k);
      const int64_t w2 = col[0], jc = col[1], c = col[2];
      const float* wrow = a.Wc + (t12 * a.wr + w2) * nin;
      const int64_t qc = a.qr[jc];
      for (int w = 0; w < a.wl; ++w) {
        const int64_t qa = qa2 - a.qwl[w];  // ket sector of a: q(a2) = q(a) + q_w
        if (qa < a.qmin || qa >= a.qmin + a.nq) continue;
        const int64_t ia = a.lsec[qa - a.qmin];
        if (ia < 0) continue;
        const int64_t rs = a.rs1[ia * a.wl + w];
        if (rs < 0) continue;
        const int64_t S = qc - qa;  // s1 + s2
        const float* t1row = a.T1 + a.t1off[ia] + (rs + a2) * a.rowlen[ia];
        for (int s1 = 0; s1 < a.d1; ++s1) {
          const int64_t s2 = S - s1;
          if (s2 < 0 || s2 >= a.d2) continue;
          const int64_t c0 = a.cs[(ia * a.d1 + s1) * a.d2 + s2];
          if (c0 < 0) continue;
          acc = fmaf(wrow[(w * a.d1 + s1) * a.d2 + s2], t1row[c0 + c], acc);
        }
      }
    }
    store_split_f<KIND>(dst, r * 2 * a.Kpl + k, a.Kpl, acc);
  }
}

// The same W-step, one block per T3 row: the row's lookups staged in shared
// memory (for every left channel w the T1 row base of (sector of a, a2) and
// q(a), the first column of every (w, s1, s2), and the combined weights Wc of
// this (t1, t2) for all w2; size wu_smem_bytes()), then each warp takes whole column runs of one
// (w2, sector of c), lanes over c, so the term loop is uniform across the
// warp (the runs are 1..~100 columns: with one thread per column the warps
// straddled runs and diverged). Same terms in the same order per element:
// bit-identical to k_u1_wsteps.
template <int KIND>
__global__ void __launch_bounds__(128) k_u1_wsteps_seg(WstepArgs a, void* __restrict__ dst) {
  extern __shared__ __align__(16) unsigned char wsm[];
  const int64_t r = blockIdx.x;
  if (r >= a.rows) return;
  const int wl = a.wl, d1 = a.d1, d2 = a.d2, wr = a.wr;
  const int nin = wl * d1 * d2;
  int64_t* base = reinterpret_cast<int64_t*>(wsm);
  int64_t* qaw = base + wl;
  int64_t* c0t = qaw + wl;
  float* wsh = reinterpret_cast<float*>(c0t + nin);
  // per warp: the current column run's terms (T1 offset, weight), in order
  const int nterm_max = wl * d1;
  int64_t* toff = reinterpret_cast<int64_t*>(wsh + wr * nin + ((wr * nin) & 1)) +
                  (threadIdx.x >> 5) * nterm_max;
  float* twt = reinterpret_cast<float*>(reinterpret_cast<int64_t*>(wsh + wr * nin + ((wr * nin) & 1)) +
                                        (blockDim.x >> 5) * nterm_max) +
               (threadIdx.x >> 5) * nterm_max;
  // the row's lookups come from tables the plan resolved on the host (two
  // dependent loads instead of a chain through the sector tables)
  const int64_t j = a.a4row[4 * r], t12 = a.a4row[4 * r + 1], ia2 = a.a4row[4 * r + 2];
  const int64_t K = a.a4kp[3 * r + 1], Kp = a.a4kp[3 * r + 2];
  for (int w = threadIdx.x; w < wl; w += blockDim.x) {
    base[w] = a.rowbase[r * wl + w];
    qaw[w] = a.ql[ia2] - a.qwl[w];
  }
  for (int i = threadIdx.x; i < nin; i += blockDim.x) c0t[i] = a.c0tab[ia2 * nin + i];
  for (int i = threadIdx.x; i < wr * nin; i += blockDim.x) wsh[i] = a.Wc[t12 * wr * nin + i];
  __syncthreads();
  for (int64_t k = K + threadIdx.x; k < Kp; k += blockDim.x)  // zero padding
    store_split_f<KIND>(dst, r * 2 * a.Kpl + k, a.Kpl, 0.0f);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int64_t s0 = a.pseg[2 * j], ns = a.pseg[2 * j + 1];
  for (int64_t sg = warp; sg < ns; sg += nwarp) {
    const int64_t* q = a.seg + 4 * (s0 + sg);
    const int64_t w2 = q[0], qc = a.qr[q[1]], k0 = q[2], len = q[3];
    const float* wrow = wsh + w2 * nin;
    // the run's terms in (w, s1) order: candidate t = w d1 + s1 on lane t % 32
    int nt = 0;
    for (int t0 = 0; t0 < nterm_max; t0 += 32) {
      const int t = t0 + lane;
      bool ok = false;
      int64_t off = 0;
      float wt = 0.0f;
      if (t < nterm_max) {
        const int w = t / d1, s1 = t % d1;
        const int64_t b = base[w];
        const int64_t s2 = qc - qaw[w] - s1;  // s1 + s2 = q(c) - q(a)
        if (b >= 0 && s2 >= 0 && s2 < d2) {
          const int64_t c0 = c0t[(w * d1 + s1) * d2 + s2];
          if (c0 >= 0) {
            ok = true;
            off = b + c0;
            wt = wrow[(w * d1 + s1) * d2 + s2];
          }
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (ok) {
        const int pos = nt + __popc(m & ((1u << lane) - 1u));
        toff[pos] = off;
        twt[pos] = wt;
      }
      nt += __popc(m);
    }
    __syncwarp();
    for (int64_t c = lane; c < len; c += 32) {
      float acc = 0.0f;
#pragma unroll 4
      for (int t = 0; t < nt; ++t) acc = fmaf(twt[t], a.T1[toff[t] + c], acc);
      store_split_f<KIND>(dst, r * 2 * a.Kpl + k0 + c, a.Kpl, acc);
    }
    __syncwarp();  // the next run overwrites this warp's term list
  }
}

size_t wu_smem_bytes(int64_t wl, int64_t d1, int64_t d2, int64_t wr) {
  const int64_t nin = wl * d1 * d2, wf = wr * nin + ((wr * nin) & 1);  // floats, even count
  const int64_t warps = 128 / 32;
  return (size_t)(2 * wl + nin) * sizeof(int64_t) + (size_t)wf * sizeof(float) +
         (size_t)warps * wl * d1 * (sizeof(int64_t) + sizeof(float));
}

// y segments from the stage-4 output blocks (zeros where a row has no K):
// one warp per row (rows hold one right sector, 1..~100 entries).
__global__ void k_u1_scatter(const double* __restrict__ Y, const int64_t* __restrict__ ysrc,
                             const int64_t* __restrict__ ydst, const int64_t* __restrict__ ylen,
                             int64_t rows, double* __restrict__ y) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const int64_t n = ylen[r], src = ysrc[r], d = ydst[r];
  for (int64_t k = threadIdx.x & 31; k < n; k += 32) y[d + k] = src >= 0 ? Y[src + k] : 0.0;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

osmps_status u1_build(osmps_u1_heff* h) {
  const int64_t nl = h->nl, nr = h->nr, d1 = h->d1, d2 = h->d2, wl = h->wl, wr = h->wr;
  std::vector<int64_t> tab;
  auto put = [&](const std::vector<int64_t>& v) {
    const int64_t off = (int64_t)tab.size();
    tab.insert(tab.end(), v.begin(), v.end());
    if (v.empty()) tab.push_back(0);  // keep every table addressable
    return off;
  };
  // sector lookup by charge (left bond)
  int64_t qmin = h->ql[0], qmax = h->ql[0];
  for (int64_t q : h->ql) { qmin = std::min(qmin, q); qmax = std::max(qmax, q); }
  h->qmin = qmin;
  h->nq = qmax - qmin + 1;
  if (h->nq > (1 << 22)) return set_error(OSMPS_EUNSUPPORTED, "u1 plan: charge range too wide");
  std::vector<int64_t> lsec(h->nq, -1);
  for (int64_t i = 0; i < nl; ++i) lsec[h->ql[i] - qmin] = i;
  // theta / y rows: per left sector, columns (s1, s2, c)
  std::vector<int64_t> rowlen(nl, 0), cs(nl * d1 * d2, -1), thoff(nl, 0);
  int64_t nth = 0;
  for (int64_t i = 0; i < nl; ++i) {
    for (int64_t s1 = 0; s1 < d1; ++s1)
      for (int64_t s2 = 0; s2 < d2; ++s2) {
        const int64_t j = find_sector(h->qr, h->ql[i] + s1 + s2);
        if (j < 0) continue;
        cs[(i * d1 + s1) * d2 + s2] = rowlen[i];
        rowlen[i] += h->chir[j];
      }
    thoff[i] = nth;
    nth += h->chil[i] * rowlen[i];
  }
  h->n_theta = nth;
  // packed L: per bra sector i2, rows a2 of segments (w, a in sector q(a2) - q_w)
  std::vector<int64_t> lrow(nl, 0), lcol(nl * wl, -1), lbase(nl, 0);
  int64_t nL = 0;
  for (int64_t i2 = 0; i2 < nl; ++i2) {
    for (int64_t w = 0; w < wl; ++w) {
      const int64_t i = find_sector(h->ql, h->ql[i2] - h->qwl[w]);
      if (i < 0) continue;
      lcol[i2 * wl + w] = lrow[i2];
      lrow[i2] += h->chil[i];
    }
    lbase[i2] = nL;
    nL += h->chil[i2] * lrow[i2];
  }
  h->n_L = nL;
  // packed R: per bra sector j2, rows c2 of segments (w, c in sector q(c2) - q_w)
  std::vector<int64_t> rrow(nr, 0), rbase(nr, 0);
  int64_t nR = 0;
  for (int64_t j2 = 0; j2 < nr; ++j2) {
    for (int64_t w = 0; w < wr; ++w) {
      const int64_t j = find_sector(h->qr, h->qr[j2] - h->qwr[w]);
      if (j >= 0) rrow[j2] += h->chir[j];
    }
    rbase[j2] = nR;
    nR += h->chir[j2] * rrow[j2];
  }
  h->n_R = nR;

  // stage 1: one problem per ket sector i
  std::vector<int64_t> rs1(nl * wl, -1), t1off(nl, 0), a1src, a1len, b1base, b1stride, b1len;
  int64_t nT1 = 0, kpmax1 = 64;
  for (int64_t i = 0; i < nl; ++i) {
    int64_t M = 0;
    for (int64_t w = 0; w < wl; ++w) {
      const int64_t i2 = find_sector(h->ql, h->ql[i] + h->qwl[w]);
      if (i2 < 0) continue;
      rs1[i * wl + w] = M;
      M += h->chil[i2];
    }
    const int64_t N = rowlen[i], K = h->chil[i];
    if (M == 0 || N == 0) {
      for (int64_t w = 0; w < wl; ++w) rs1[i * wl + w] = -1;
      continue;
    }
    GroupProblem p = {};
    p.a_row0 = (int)a1src.size();
    p.b_row0 = (int)b1base.size();
    p.M = (int)M;
    p.N = (int)N;
    p.c_off = nT1;
    p.ldc = N;
    t1off[i] = nT1;
    for (int64_t w = 0; w < wl; ++w) {
      const int64_t i2 = find_sector(h->ql, h->ql[i] + h->qwl[w]);
      if (i2 < 0) continue;
      for (int64_t a2 = 0; a2 < h->chil[i2]; ++a2) {
        a1src.push_back(lbase[i2] + a2 * lrow[i2] + lcol[i2 * wl + w]);
        a1len.push_back(K);
      }
    }
    for (int64_t n = 0; n < N; ++n) {
      b1base.push_back(thoff[i] + n);
      b1stride.push_back(N);
      b1len.push_back(K);
    }
    nT1 += M * N;
    h->p1.push_back(p);
    h->kp1.push_back(round_up(K, 64));
    kpmax1 = std::max(kpmax1, round_up(K, 64));
    h->flops1 += 2.0 * (double)M * (double)N * (double)K;
  }
  h->rowsA1 = (int64_t)a1src.size();
  h->rowsB1 = (int64_t)b1base.size();
  h->Kpl1 = kpmax1;
  h->n_T1 = nT1;

  // stage 4: one problem per output sector j of c2
  std::vector<int64_t> a4row, a4col, a4kp, b4src, b4len, ysrc, ydst, ylen, seg, pseg;
  int64_t nY = 0, kpmax4 = 64, ncol = 0;
  for (int64_t j = 0; j < nr; ++j) {
    const int64_t colbase = ncol;
    int64_t K = 0;
    pseg.push_back((int64_t)seg.size() / 4);
    for (int64_t w2 = 0; w2 < wr; ++w2) {
      const int64_t jc = find_sector(h->qr, h->qr[j] - h->qwr[w2]);
      if (jc < 0) continue;
      seg.push_back(w2);
      seg.push_back(jc);
      seg.push_back(K);
      seg.push_back(h->chir[jc]);
      for (int64_t c = 0; c < h->chir[jc]; ++c) {
        a4col.push_back(w2);
        a4col.push_back(jc);
        a4col.push_back(c);
      }
      K += h->chir[jc];
    }
    ncol += K;
    pseg.push_back((int64_t)seg.size() / 4 - pseg.back());
    const int64_t Kp = K > 0 ? round_up(K, 64) : 0;
    const int64_t N = h->chir[j];
    const int64_t row0 = (int64_t)ylen.size();
    for (int64_t t1 = 0; t1 < d1; ++t1)
      for (int64_t t2 = 0; t2 < d2; ++t2) {
        const int64_t ia2 = find_sector(h->ql, h->qr[j] - t1 - t2);
        if (ia2 < 0) continue;
        const int64_t cseg = cs[(ia2 * d1 + t1) * d2 + t2];
        for (int64_t a2 = 0; a2 < h->chil[ia2]; ++a2) {
          a4row.push_back(j);
          a4row.push_back(t1 * d2 + t2);
          a4row.push_back(ia2);
          a4row.push_back(a2);
          a4kp.push_back(colbase);
          a4kp.push_back(K);
          a4kp.push_back(Kp);
          ydst.push_back(thoff[ia2] + a2 * rowlen[ia2] + cseg);
          ylen.push_back(N);
          ysrc.push_back(-1);
        }
      }
    const int64_t M = (int64_t)ylen.size() - row0;
    if (M == 0 || K == 0) continue;  // rows (if any) stay zero in y
    h->n_A4 += M * K;
    GroupProblem p = {};
    p.a_row0 = (int)row0;
    p.b_row0 = (int)b4src.size();
    p.M = (int)M;
    p.N = (int)N;
    p.c_off = nY;
    p.ldc = N;
    for (int64_t r = 0; r < M; ++r) ysrc[row0 + r] = nY + r * N;
    for (int64_t c2 = 0; c2 < N; ++c2) {
      b4src.push_back(rbase[j] + c2 * rrow[j]);
      b4len.push_back(rrow[j]);
    }
    nY += M * N;
    h->p4.push_back(p);
    h->kp4.push_back(Kp);
    kpmax4 = std::max(kpmax4, Kp);
    h->flops4 += 2.0 * (double)M * (double)N * (double)K;
  }
  h->rowsA4 = (int64_t)ylen.size();
  h->rowsB4 = (int64_t)b4src.size();
  // the W-step's per-row and per-sector lookups, resolved once: for T3 row r
  // (sector ia2 of a2, a2 within it) and left channel w, the T1 row of the
  // ket sector q(a2) - q_w; for sector ia2, the first T1 column of (s1, s2)
  auto ket_sector = [&](int64_t qa) {
    return (qa >= h->qmin && qa < h->qmin + h->nq) ? lsec[qa - h->qmin] : (int64_t)-1;
  };
  const int64_t nin = wl * d1 * d2;
  std::vector<int64_t> rowbase((size_t)std::max<int64_t>(h->rowsA4 * wl, 1), -1);
  for (int64_t r = 0; r < h->rowsA4; ++r) {
    const int64_t ia2 = a4row[4 * r + 2], a2 = a4row[4 * r + 3];
    for (int64_t w = 0; w < wl; ++w) {
      const int64_t ia = ket_sector(h->ql[ia2] - h->qwl[w]);
      if (ia < 0) continue;
      const int64_t rs = rs1[ia * wl + w];
      if (rs >= 0) rowbase[r * wl + w] = t1off[ia] + (rs + a2) * rowlen[ia];
    }
  }
  std::vector<int64_t> c0tab((size_t)std::max<int64_t>(nl * nin, 1), -1);
  for (int64_t ia2 = 0; ia2 < nl; ++ia2)
    for (int64_t i = 0; i < nin; ++i) {
      const int64_t w = i / (d1 * d2), ss = i % (d1 * d2);
      const int64_t ia = ket_sector(h->ql[ia2] - h->qwl[w]);
      if (ia >= 0) c0tab[ia2 * nin + i] = cs[ia * d1 * d2 + ss];
    }
  h->Kpl4 = kpmax4;
  h->n_Y = nY;
  if (h->rowsA1 > (1 << 30) || h->rowsB1 > (1 << 30) || h->rowsA4 > 65535 || nth > ((int64_t)1 << 40))
    return set_error(OSMPS_EUNSUPPORTED, "u1 plan: block structure too large");
  h->tiles1 = group_tiles(h->p1.data(), (int)h->p1.size(), 256);
  h->tiles4 = group_tiles(h->p4.data(), (int)h->p4.size(), 256);

  h->t_lsec = put(lsec);
  h->t_ql = put(h->ql);
  h->t_qr = put(h->qr);
  h->t_qwl = put(h->qwl);
  h->t_rowlen = put(rowlen);
  h->t_t1off = put(t1off);
  h->t_rs1 = put(rs1);
  h->t_cs = put(cs);
  h->t_a1src = put(a1src);
  h->t_a1len = put(a1len);
  h->t_b1base = put(b1base);
  h->t_b1stride = put(b1stride);
  h->t_b1len = put(b1len);
  h->t_a4row = put(a4row);
  h->t_a4col = put(a4col);
  h->t_a4kp = put(a4kp);
  h->t_seg = put(seg);
  h->t_rowbase = put(rowbase);
  h->t_c0tab = put(c0tab);
  h->t_pseg = put(pseg);
  h->t_b4src = put(b4src);
  h->t_b4len = put(b4len);
  h->t_ysrc = put(ysrc);
  h->t_ydst = put(ydst);
  h->t_ylen = put(ylen);
  OSMPS_CUDA(cudaMalloc(&h->d_tab, tab.size() * sizeof(int64_t)));
  OSMPS_CUDA(cudaMemcpy(h->d_tab, tab.data(), tab.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  const size_t np = std::max<size_t>(1, h->p1.size() + h->p4.size());
  OSMPS_CUDA(cudaMalloc(&h->d_prob, np * sizeof(GroupProblem)));
  // buffers (operand element size up to 4 bytes: tf32)
  size_t o = 0;
  h->o_A1 = o; o = align256(o + (size_t)std::max<int64_t>(h->rowsA1, 1) * 2 * h->Kpl1 * 4);
  h->o_B1 = o; o = align256(o + (size_t)std::max<int64_t>(h->rowsB1, 1) * 2 * h->Kpl1 * 4);
  h->o_T1 = o; o = align256(o + (size_t)std::max<int64_t>(nT1, 1) * 4);
  h->o_A4 = o; o = align256(o + (size_t)std::max<int64_t>(h->rowsA4, 1) * 2 * h->Kpl4 * 4);
  h->o_B4 = o; o = align256(o + (size_t)std::max<int64_t>(h->rowsB4, 1) * 2 * h->Kpl4 * 4);
  h->o_Wc = o; o = align256(o + (size_t)(wl * d1 * d2) * (d1 * d2 * wr) * 4);
  h->o_Y = o; o = align256(o + (size_t)std::max<int64_t>(nY, 1) * 8);
  OSMPS_CUDA(cudaMalloc(&h->d_buf, o));
  return OSMPS_OK;
}

template <int KIND>
osmps_status u1_prepare_kind(osmps_u1_heff* h, const double* L, const double* W1, const double* W2,
                             const double* R, cudaStream_t s) {
  const int64_t* T = h->d_tab;
  uint8_t* B = h->d_buf;
  if (h->kind_loaded != KIND) {
    // K slices per problem depend on the operand type (128 bytes of K per slice)
    const int kelem = KIND == TC_BF16 ? 64 : 32;
    // kept in the host tables too: a table rebuilt for another tile width is
    // uploaded from them
    for (size_t i = 0; i < h->p1.size(); ++i) h->p1[i].nkb = (int)(h->kp1[i] / kelem);
    for (size_t i = 0; i < h->p4.size(); ++i) h->p4[i].nkb = (int)(h->kp4[i] / kelem);
    std::vector<GroupProblem> all(h->p1);
    all.insert(all.end(), h->p4.begin(), h->p4.end());
    OSMPS_CUDA(cudaStreamSynchronize(s));  // earlier launches may still read the table
    if (!all.empty())
      OSMPS_CUDA(cudaMemcpy(h->d_prob, all.data(), all.size() * sizeof(GroupProblem),
                            cudaMemcpyHostToDevice));
    h->kind_loaded = KIND;
  }
  // L and R as split operands, combined W coefficients
  if (h->rowsA1 > 0) {
    k_row_gather_split<KIND><<<ew_grid(h->rowsA1 * h->Kpl1), 256, 0, s>>>(
        L, T + h->t_a1src, T + h->t_a1len, h->rowsA1, h->Kpl1, B + h->o_A1);
    note_launch();
  }
  if (h->rowsB4 > 0) {
    k_row_gather_split<KIND><<<ew_grid(h->rowsB4 * h->Kpl4), 256, 0, s>>>(
        R, T + h->t_b4src, T + h->t_b4len, h->rowsB4, h->Kpl4, B + h->o_B4);
    note_launch();
  }
  { k_wcomb<<<ew_grid(h->wl * h->d1 * h->d2 * h->d1 * h->d2 * h->wr), 256, 0, s>>>(
        W1, W2, (int)h->d1, (int)h->d2, (int)h->wl, (int)h->wm, (int)h->wr,
        reinterpret_cast<float*>(B + h->o_Wc)); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  h->prepared_kind = KIND;
  return OSMPS_OK;
}

// Rebuild and upload stage st's problem table for tile width bn.
osmps_status u1_table_width(osmps_u1_heff* h, int st, int bn, cudaStream_t s) {
  std::vector<GroupProblem>& p = st == 1 ? h->p1 : h->p4;
  int& cur = st == 1 ? h->bn1 : h->bn4;
  if (cur == bn || p.empty()) return OSMPS_OK;
  (st == 1 ? h->tiles1 : h->tiles4) = group_tiles(p.data(), (int)p.size(), bn);
  GroupProblem* dst = h->d_prob + (st == 1 ? 0 : h->p1.size());
  OSMPS_CUDA(cudaMemcpyAsync(dst, p.data(), p.size() * sizeof(GroupProblem), cudaMemcpyHostToDevice, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));  // the host table is rebuilt in place next time
  cur = bn;
  return OSMPS_OK;
}

// One grouped stage with its settled tile width: on the plan's first product
// outside capture, the width comes from the context's tuning table for the
// stage's size class, or is measured (all three widths, the fastest kept).
osmps_status u1_grouped(osmps_ctx* ctx, osmps_u1_heff* h, int st, GemmTcGrouped g, cudaStream_t s) {
  bool& settled = st == 1 ? h->settled1 : h->settled4;
  std::vector<GroupProblem>& p = st == 1 ? h->p1 : h->p4;
  if (!settled && !ctx->capturing) {
    int64_t t64 = 0;
    for (const GroupProblem& q : p) t64 += cdiv(q.M, 128) * cdiv(q.N, 64);
    const TcKey key = tc_key(1, g.kind, g.out, (int64_t)p.size(), t64, cdiv(g.Kpl, 512));
    int bn = tc_tuned_width(ctx, key);
    if (bn == 0 && tc_may_tune(ctx)) {
      const int widths[3] = {256, 128, 64};
      float us[3] = {0.f, 0.f, 0.f};
      for (int w = 0; w < 3; ++w) {
        OSMPS_TRY(u1_table_width(h, st, widths[w], s));
        g.bn = widths[w];
        g.n_tiles = st == 1 ? h->tiles1 : h->tiles4;
        OSMPS_TRY(gemm_tc_grouped(ctx, g, s));
        OSMPS_TRY(tc_time_launches(ctx, s, 2, &us[w], [&](cudaStream_t q) { return gemm_tc_grouped(ctx, g, q); }));
      }
      bn = tc_record_tuning(ctx, key, widths, us);
    }
    if (bn == 0) bn = 256;
    OSMPS_TRY(u1_table_width(h, st, bn, s));
    settled = true;
  }
  g.bn = st == 1 ? h->bn1 : h->bn4;
  g.n_tiles = st == 1 ? h->tiles1 : h->tiles4;
  return gemm_tc_grouped(ctx, g, s);
}

template <int KIND>
osmps_status u1_apply_kind(osmps_ctx* ctx, osmps_u1_heff* h, const double* theta, double* y,
                           cudaStream_t s) {
  const int64_t* T = h->d_tab;
  uint8_t* B = h->d_buf;
  // stage 1
  if (h->rowsB1 > 0) {
    dim3 grid((unsigned)cdiv(h->rowsB1, 32), (unsigned)cdiv(h->Kpl1, 32));
    k_theta_split<KIND><<<grid, dim3(32, 8), 0, s>>>(theta, T + h->t_b1base, T + h->t_b1stride,
                                                     T + h->t_b1len, h->rowsB1, h->Kpl1, B + h->o_B1);
    note_launch();
  }
  OSMPS_LAUNCH_CHECK();
  if (!h->p1.empty()) {
    GemmTcGrouped g;
    g.kind = KIND;
    g.out = TC_OUT_F32;
    g.A = B + h->o_A1;
    g.rowsA = h->rowsA1;
    g.B = B + h->o_B1;
    g.rowsB = h->rowsB1;
    g.Kpl = h->Kpl1;
    g.C = B + h->o_T1;
    g.probs = h->d_prob;
    g.n_prob = (int)h->p1.size();
    g.logical_flops = h->flops1;
    OSMPS_TRY(u1_grouped(ctx, h, 1, g, s));
  }
  // stages 2 + 3
  if (h->rowsA4 > 0) {
    WstepArgs a;
    a.T1 = reinterpret_cast<const float*>(B + h->o_T1);
    a.Wc = reinterpret_cast<const float*>(B + h->o_Wc);
    a.lsec = T + h->t_lsec;
    a.ql = T + h->t_ql;
    a.qr = T + h->t_qr;
    a.qwl = T + h->t_qwl;
    a.rowlen = T + h->t_rowlen;
    a.t1off = T + h->t_t1off;
    a.rs1 = T + h->t_rs1;
    a.cs = T + h->t_cs;
    a.a4row = T + h->t_a4row;
    a.a4col = T + h->t_a4col;
    a.a4kp = T + h->t_a4kp;
    a.seg = T + h->t_seg;
    a.pseg = T + h->t_pseg;
    a.rowbase = T + h->t_rowbase;
    a.c0tab = T + h->t_c0tab;
    a.rows = h->rowsA4;
    a.Kpl = h->Kpl4;
    a.qmin = h->qmin;
    a.nq = h->nq;
    a.d1 = (int)h->d1;
    a.d2 = (int)h->d2;
    a.wl = (int)h->wl;
    a.wr = (int)h->wr;
    dim3 grid((unsigned)std::max<int64_t>(1, cdiv(h->Kpl4, 256)), (unsigned)h->rowsA4);
    const size_t sm = wu_smem_bytes(h->wl, h->d1, h->d2, h->wr);
    // algorithmic bytes: T1 read once (float32), the split operand's entries
    // written once (two pieces of 2 or 4 bytes)
    const double wbytes = 4.0 * (double)h->n_T1 +
                          (KIND == TC_BF16 ? 4.0 : 8.0) * (double)h->n_A4;
    const int ph = prof_begin(s);
    if (sm <= 48 * 1024)
      k_u1_wsteps_seg<KIND><<<(unsigned)h->rowsA4, 128, sm, s>>>(a, B + h->o_A4);
    else
      k_u1_wsteps<KIND><<<grid, 256, 0, s>>>(a, B + h->o_A4);
    note_launch();
    prof_end(ph, s, OSMPS_KERNEL_U1_WSTEP, wbytes, 0.0);
    OSMPS_LAUNCH_CHECK();
  }
  // stage 4
  if (!h->p4.empty()) {
    GemmTcGrouped g;
    g.kind = KIND;
    g.out = TC_OUT_F64;
    g.A = B + h->o_A4;
    g.rowsA = h->rowsA4;
    g.B = B + h->o_B4;
    g.rowsB = h->rowsB4;
    g.Kpl = h->Kpl4;
    g.C = B + h->o_Y;
    g.probs = h->d_prob + h->p1.size();
    g.n_prob = (int)h->p4.size();
    g.logical_flops = h->flops4;
    OSMPS_TRY(u1_grouped(ctx, h, 4, g, s));
  }
  if (h->rowsA4 > 0) {
    k_u1_scatter<<<(unsigned)cdiv(h->rowsA4, 8), 256, 0, s>>>(reinterpret_cast<const double*>(B + h->o_Y), T + h->t_ysrc,
                                      T + h->t_ydst, T + h->t_ylen, h->rowsA4, y);
    note_launch();
    OSMPS_LAUNCH_CHECK();
  }
  return OSMPS_OK;
}

}  // namespace
}  // namespace osmps

using namespace osmps;

extern "C" {

osmps_status osmps_u1_heff_create(osmps_ctx* ctx, const osmps_u1_desc* d, osmps_u1_heff** out) {
  clear_error();
  if (!ctx || !d || !out) return set_error(OSMPS_EINVAL, "osmps_u1_heff_create: null argument");
  *out = nullptr;
  if (d->n_left < 1 || d->n_right < 1 || d->d1 < 1 || d->d2 < 1 || d->wl < 1 || d->wm < 1 ||
      d->wr < 1 || d->d1 > 64 || d->d2 > 64 || d->wl > 64 || d->wm > 64 || d->wr > 64)
    return set_error(OSMPS_ESHAPE, "osmps_u1_heff_create: bad sizes");
  if (!d->q_left || !d->chi_left || !d->q_right || !d->chi_right || !d->q_wl || !d->q_wr)
    return set_error(OSMPS_EINVAL, "osmps_u1_heff_create: null table");
  static std::atomic<uint64_t> next_uid{1};
  osmps_u1_heff* h = new osmps_u1_heff();
  h->uid = next_uid.fetch_add(1);
  h->ctx = ctx;
  h->nl = d->n_left;
  h->nr = d->n_right;
  h->d1 = d->d1;
  h->d2 = d->d2;
  h->wl = d->wl;
  h->wm = d->wm;
  h->wr = d->wr;
  h->ql.assign(d->q_left, d->q_left + d->n_left);
  h->chil.assign(d->chi_left, d->chi_left + d->n_left);
  h->qr.assign(d->q_right, d->q_right + d->n_right);
  h->chir.assign(d->chi_right, d->chi_right + d->n_right);
  h->qwl.assign(d->q_wl, d->q_wl + d->wl);
  h->qwr.assign(d->q_wr, d->q_wr + d->wr);
  osmps_status st = OSMPS_OK;
  for (int64_t c : h->chil) if (c < 1) st = OSMPS_ESHAPE;
  for (int64_t c : h->chir) if (c < 1) st = OSMPS_ESHAPE;
  for (size_t i = 0; i < h->ql.size(); ++i)
    for (size_t j = 0; j < i; ++j) if (h->ql[i] == h->ql[j]) st = OSMPS_EINVAL;
  for (size_t i = 0; i < h->qr.size(); ++i)
    for (size_t j = 0; j < i; ++j) if (h->qr[i] == h->qr[j]) st = OSMPS_EINVAL;
  if (st != OSMPS_OK) {
    delete h;
    return set_error(st, "osmps_u1_heff_create: sector sizes must be >= 1 and charges distinct per bond");
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess || (st = u1_build(h)) != OSMPS_OK) {
    if (st == OSMPS_OK) st = set_error(OSMPS_ECUDA, "osmps_u1_heff_create: cudaSetDevice failed");
    osmps_u1_heff_destroy(h);
    return st;
  }
  *out = h;
  return OSMPS_OK;
}

osmps_status osmps_u1_heff_destroy(osmps_u1_heff* h) {
  if (!h) return OSMPS_OK;
  cudaSetDevice(h->ctx->device);
  cudaDeviceSynchronize();
  if (h->d_tab) cudaFree(h->d_tab);
  if (h->d_prob) cudaFree(h->d_prob);
  if (h->d_buf) cudaFree(h->d_buf);
  delete h;
  return OSMPS_OK;
}

osmps_status osmps_u1_heff_sizes(const osmps_u1_heff* h, int64_t* n_theta, int64_t* n_L,
                                 int64_t* n_R, double* flops) {
  clear_error();
  if (!h) return set_error(OSMPS_EINVAL, "osmps_u1_heff_sizes: null handle");
  if (n_theta) *n_theta = h->n_theta;
  if (n_L) *n_L = h->n_L;
  if (n_R) *n_R = h->n_R;
  if (flops) *flops = h->flops1 + h->flops4;
  return OSMPS_OK;
}

osmps_status osmps_u1_heff_stage_sizes(const osmps_u1_heff* h, int64_t* n_t1, int64_t* n_a4,
                                       int64_t* n_y) {
  clear_error();
  if (!h) return set_error(OSMPS_EINVAL, "osmps_u1_heff_stage_sizes: null handle");
  if (n_t1) *n_t1 = h->n_T1;
  if (n_a4) *n_a4 = h->n_A4;
  if (n_y) *n_y = h->n_Y;
  return OSMPS_OK;
}

osmps_status osmps_u1_heff_prepare(osmps_ctx* ctx, osmps_u1_heff* h, const double* L,
                                   const double* W1, const double* W2, const double* R,
                                   int precision, void* stream) {
  clear_error();
  if (!ctx || !h || !L || !W1 || !W2 || !R)
    return set_error(OSMPS_EINVAL, "osmps_u1_heff_prepare: null argument");
  if (precision != OSMPS_PREC_BF16X3 && precision != OSMPS_PREC_TF32X3)
    return set_error(OSMPS_EUNSUPPORTED, "osmps_u1_heff_prepare: precision %d (bf16x3 or tf32x3)", precision);
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == OSMPS_PREC_BF16X3) return u1_prepare_kind<TC_BF16>(h, L, W1, W2, R, s);
  return u1_prepare_kind<TC_TF32>(h, L, W1, W2, R, s);
}

osmps_status osmps_u1_heff_apply(osmps_ctx* ctx, osmps_u1_heff* h, const double* theta, double* y,
                                 void* stream) {
  clear_error();
  if (!ctx || !h || !theta || !y) return set_error(OSMPS_EINVAL, "osmps_u1_heff_apply: null argument");
  if (y == theta) return set_error(OSMPS_EINVAL, "osmps_u1_heff_apply: y aliases theta");
  if (h->prepared_kind < 0) return set_error(OSMPS_EINVAL, "osmps_u1_heff_apply: no prepared operator");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  if (h->prepared_kind == TC_BF16) return u1_apply_kind<TC_BF16>(ctx, h, theta, y, s);
  return u1_apply_kind<TC_TF32>(ctx, h, theta, y, s);
}

osmps_status osmps_lanczos_ground_u1(osmps_ctx* ctx, osmps_u1_heff* h, const double* L,
                                     const double* W1, const double* W2, const double* R,
                                     double* theta_inout, int max_iter, double tol, int precision,
                                     double* energy_out, int* iters_out, double* resid_out,
                                     void* stream) {
  clear_error();
  if (!ctx || !h || !L || !W1 || !W2 || !R || !theta_inout || !energy_out || !iters_out)
    return set_error(OSMPS_EINVAL, "osmps_lanczos_ground_u1: null argument");
  if (max_iter < 1 || max_iter > 512)
    return set_error(OSMPS_EINVAL, "osmps_lanczos_ground_u1: max_iter %d outside [1, 512]", max_iter);
  if (!(tol >= 0.0)) return set_error(OSMPS_EINVAL, "osmps_lanczos_ground_u1: tol %g", tol);
  if (h->n_theta < 1) return set_error(OSMPS_ESHAPE, "osmps_lanczos_ground_u1: empty sector");
  OSMPS_TRY(osmps_u1_heff_prepare(ctx, h, L, W1, W2, R, precision, stream));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  const Matvec mv = [&](const double* x, double* y, cudaStream_t q) {
    return h->prepared_kind == TC_BF16 ? u1_apply_kind<TC_BF16>(ctx, h, x, y, q)
                                       : u1_apply_kind<TC_TF32>(ctx, h, x, y, q);
  };
  const long long key[3] = {2, (long long)h->uid, (long long)h->prepared_kind};
  return lanczos_core(ctx, h->n_theta, theta_inout, max_iter, tol, mv, energy_out, iters_out,
                      resid_out, s, nullptr, 0, 0, key, 3);
}

osmps_status osmps_heff_apply_u1(osmps_ctx* ctx, osmps_u1_heff* h, const double* L,
                                 const double* W1, const double* W2, const double* R,
                                 const double* theta, double* y, int precision, void* stream) {
  clear_error();
  if (!ctx || !h || !L || !W1 || !W2 || !R || !theta || !y)
    return set_error(OSMPS_EINVAL, "osmps_heff_apply_u1: null argument");
  if (y == theta) return set_error(OSMPS_EINVAL, "osmps_heff_apply_u1: y aliases theta");
  if (precision != OSMPS_PREC_BF16X3 && precision != OSMPS_PREC_TF32X3)
    return set_error(OSMPS_EUNSUPPORTED, "osmps_heff_apply_u1: precision %d (bf16x3 or tf32x3)", precision);
  OSMPS_TRY(osmps_u1_heff_prepare(ctx, h, L, W1, W2, R, precision, stream));
  return osmps_u1_heff_apply(ctx, h, theta, y, stream);
}

}  // extern "C"
