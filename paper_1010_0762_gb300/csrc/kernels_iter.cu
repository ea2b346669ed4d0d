// kernels_iter.cu -- the per-iteration kernels of Algorithm 2 (RBiCG), the initial projection
// of eq. (minusXR), the final correction of step 7, the true residual, the random restart of
// step 3 and the construction of A^H.
//
// One iteration i = three grid-wide passes (two without a recycle space, where phase 1 also
// does phase 2's reduction), each ending in a deterministic grid reduction whose finishing block
// writes the scalars of the next pass into DevState:
//   phase 1: p_i = r_{i-1} + beta_{i-1} p_{i-1}, pt_i likewise (formed while gathering),
//            z_i = Op p_i, zt_i = Op^H pt_i, and the projections
//            zeta_i = D_c^{-1} Ct^H z_i, zetat_i = D_c^{-1} C^H zt_i        (eq. (CcheckChat))
//   phase 2: q_i = z_i - C zeta_i, qt_i = zt_i - Ct zetat_i, (pt_i, q_i) -> alpha_i,
//            zeta_c += alpha zeta, zetat_c += conj(alpha) zetat
//   phase 3: x_i, xt_i, r_i, rt_i updates, rho_i = (rt_i, r_i), ||r_i||, ||rt_i||,
//            stopping test, beta_i = rho_i / rho_{i-1}
#include <algorithm>
#include <cstdlib>

#include "internal.cuh"

namespace rb {

// ------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ zd ld_cg(const zd* p) {
  const double* q = reinterpret_cast<const double*>(p);
  return zd(__ldcg(q), __ldcg(q + 1));
}

// A block's place in its solve: block `id` of `n`.  A single solve uses (blockIdx.x, gridDim.x);
// a batched launch deals consecutive block ranges to its requests, so every request sees the
// same blocks, partial sums and reduction order as when it runs alone.
struct Blk {
  int id, n;
};

// Returns true in every thread of the block that arrives last at `cnt` (after all other
// blocks' partial writes are visible); the last block resets the counter.  The barrier orders
// the block's writes before thread 0's fence, which publishes them before the arrival; the last
// block's thread 0 fences again before its threads read the others' rows.
__device__ __forceinline__ bool arrive_last(unsigned int* cnt, int nblk) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(cnt, 1u);
    const int last = t == (unsigned int)nblk - 1;
    if (last) {
      *cnt = 0u;
      __threadfence();
    }
    s_last = last;
  }
  __syncthreads();
  return s_last;
}

// Programmatic dependent launch.  A phase kernel launched with programmatic stream
// serialization may be scheduled while the kernel before it in the stream finishes its
// reduction tail; pdl_wait() holds it until that kernel has completed and its writes are
// visible, so it comes before the first access to anything the previous kernel wrote.
// pdl_release() lets the next kernel be scheduled once every block of this one has passed it.
// Without that launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Block sums of three per-thread values with fewer FP64 adds than three shuffle trees: in each
// warp a reduce-scatter butterfly (offset 16 splits the values between the lane halves, offset 8
// between quarters, offsets 4, 2, 1 finish one value per group of 8 lanes: 6 adds a lane instead
// of 15), then the warps' results in warp order.  Fixed order throughout.  out[0..2] (shared)
// holds the totals on return; smem holds NTHREADS / 32 * 4 values.
template <class A>
__device__ void block_sum3(A v0, A v1, A v2, A* smem, A* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool h16 = lane & 16, h8 = lane & 8;
  const A z = A(0.0);
  A k0 = h16 ? v2 : v0, k1 = h16 ? z : v1;
  const A s0 = h16 ? v0 : v2, s1 = h16 ? v1 : z;
  k0 += shfl_xor(s0, 16);
  k1 += shfl_xor(s1, 16);
  A r = h8 ? k1 : k0;
  r += shfl_xor(h8 ? k0 : k1, 8);
  r += shfl_xor(r, 4);
  r += shfl_xor(r, 2);
  r += shfl_xor(r, 1);
  // lane 0: v0, lane 8: v1, lane 16: v2 (lane 24 holds the zero pad)
  if ((lane & 7) == 0 && lane < 24) smem[warp * 4 + (lane >> 3)] = r;
  __syncthreads();
  if (threadIdx.x < 3) {
    A t = smem[threadIdx.x];
    for (int w = 1; w < NTHREADS / 32; ++w) t += smem[w * 4 + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// Sum part[b * cnt + c] over b = 0..G-1 for every column c (fixed order: lane-strided per
// warp, then a fixed shuffle tree); out (shared) receives cnt values.
template <class A>
__device__ void reduce_cols(const A* part, int G, int cnt, A* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = w; c < cnt; c += nw) {
    A s = A(0.0);
    for (int b = lane; b < G; b += 32) s += ld_cg(part + (int64_t)b * cnt + c);
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
  }
  __syncthreads();
}

// Block-sum `cnt` accumulators (register arrays) and write them as this block's row of part.
template <class A>
__device__ void write_partials(A* vals, int cnt, A* smem, A* part, int bid) {
  block_sum_vec(vals, cnt, smem);
  if (threadIdx.x < cnt) part[(int64_t)bid * cnt + threadIdx.x] = smem[threadIdx.x];
}

// Rows [r0, r1) of block g of a solve: a contiguous range of whole 32-row chunks, the chunk
// count split as evenly as it divides.  With a grid that is a multiple of the blocks resident
// on the GPU, every SM then receives the same number of rows.
__device__ __forceinline__ void block_rows(int n, Blk g, int& r0, int& r1) {
  const int64_t nch = (n + 31) >> 5;
  r0 = (int)((nch * g.id / g.n) << 5);
  const int e = (int)((nch * (g.id + 1) / g.n) << 5);
  r1 = e < n ? e : n;
}

// Sum CNT columns over `nrows` rows of `rows` (row stride CNT) in a fixed order: lane-strided
// per warp, then the fixed shuffle tree.  out (shared) receives the CNT sums.
template <class A, int CNT>
__device__ void sum_rows(const A* rows, int nrows, A* out) {
  constexpr int NW = NTHREADS / 32;
  constexpr int CPW = (CNT + NW - 1) / NW;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  A acc[CPW];
#pragma unroll
  for (int u = 0; u < CPW; ++u) acc[u] = A(0.0);
  for (int b = lane; b < nrows; b += 32) {
#pragma unroll
    for (int u = 0; u < CPW; ++u)
      if (w + NW * u < CNT) acc[u] += ld_cg(rows + (int64_t)b * CNT + w + NW * u);
  }
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    const A t = warp_sum(acc[u]);
    if (lane == 0 && w + NW * u < CNT) out[w + NW * u] = t;
  }
  __syncthreads();
}

// Deterministic two-level grid reduction of CNT values per block.  The blocks of a solve form
// groups of consecutive ids (group_size); the last block of a group to arrive sums the group's
// rows in id order, and the last group to finish sums the group rows in group order.  So the
// result does not depend on arrival order, and the critical path after the last arrival is two
// short L2 round trips instead of one block reading every block's row.  `tot` (shared) holds
// this block's CNT totals on entry; the function returns true only in the block that finishes,
// with the grand totals in `tot`.  part: g.n rows, then group_count(g.n) rows, CNT wide.
template <class A, int CNT>
__device__ bool grid_reduce(A* tot, A* part, unsigned int* ctr, Blk g) {
  const int gs = group_size(g.n), ng = (g.n + gs - 1) / gs;
  const int grp = g.id / gs, b0 = grp * gs;
  const int gsz = g.n - b0 < gs ? g.n - b0 : gs;
  A* gpart = part + (int64_t)g.n * CNT;
  if (threadIdx.x < CNT) part[(int64_t)g.id * CNT + threadIdx.x] = tot[threadIdx.x];
  if (!arrive_last(&ctr[grp], gsz)) return false;
  sum_rows<A, CNT>(part + (int64_t)b0 * CNT, gsz, tot);
  if (threadIdx.x < CNT) gpart[(int64_t)grp * CNT + threadIdx.x] = tot[threadIdx.x];
  if (!arrive_last(&ctr[GMAX], ng)) return false;
  sum_rows<A, CNT>(gpart, ng, tot);
  return true;
}

// Deterministic one-level grid reduction of three values per block (the iteration scalars):
// every block writes its row, the last to arrive sums all rows -- thread t the rows t, t + 256,
// ..., one round of independent loads -- and combines the threads' sums with block_sum3.  One
// arrival instead of the two of grid_reduce: for three values the rows of all blocks are few
// enough to read at once.  tot and red as in block_sum3; the grand totals land in tot.
template <class A>
__device__ bool grid_reduce3(A* tot, A* red, A* part, unsigned int* ctr, Blk g) {
  if (threadIdx.x < 3) part[(int64_t)g.id * 3 + threadIdx.x] = tot[threadIdx.x];
  if (!arrive_last(&ctr[GMAX], g.n)) return false;
  A s0 = A(0.0), s1 = A(0.0), s2 = A(0.0);
  for (int b = threadIdx.x; b < g.n; b += NTHREADS) {
    s0 += ld_cg(part + (int64_t)b * 3);
    s1 += ld_cg(part + (int64_t)b * 3 + 1);
    s2 += ld_cg(part + (int64_t)b * 3 + 2);
  }
  block_sum3(s0, s1, s2, red, tot);
  return true;
}

// The three sums of one row that decide alpha_i: (pt_i, q_i), ||q_i||^2, ||pt_i||^2.
template <class A, class T>
__device__ __forceinline__ void alpha_terms(A& pq, A& nq, A& npt, T ptr, T q) {
  pq += cmul(cvt<A>(ptr), cvt<A>(q));
  nq += A((double)abs2(q));
  npt += A((double)abs2(ptr));
}

// In the block that finished the (pt, q) reduction (tot = the three sums): alpha_i =
// rho_{i-1} / (pt_i, q_i) with the finiteness and breakdown tests, then zeta_c += alpha zeta
// and zetat_c += conj(alpha) zetat for the k recycle columns (Algorithm 2).
// rho_prev: st->rho, read at the start of the kernel (it does not change during it).
template <class A>
__device__ void finish_alpha(DevState* st, const A* tot, int i, int k, zd rho_prev) {
  __shared__ int s_stop;
  if (threadIdx.x == 0) {
    const zd PQ = to_zd(tot[0]);
    const double NQ = real_of(tot[1]), NPT = real_of(tot[2]);
    int stop = 0;
    if (!isfinite(PQ.re) || !isfinite(PQ.im) || !isfinite(NQ) || !isfinite(NPT)) {
      stop = DONE_NONFINITE;
    } else if (abs2(PQ) <= (BREAKDOWN_EPS * NQ) * (BREAKDOWN_EPS * NPT)) {   // |PQ| <= eps ||q|| ||pt||
      stop = DONE_BREAK_PQ;
    } else {
      const zd al = rho_prev * crcp(PQ);
      st->alpha = al;
      st->h_alpha[i % HR] = al;
    }
    if (stop) st->done = stop;
    s_stop = stop;
  }
  __syncthreads();
  if (s_stop) return;
  if (threadIdx.x < k) {
    const zd al = st->alpha;
    const int c = threadIdx.x;
    const zd zc = st->zeta[c], ztc = st->zetat[c];
    st->zeta_c[c] += al * zc;
    st->zetat_c[c] += conjg(al) * ztc;
    st->h_zeta[i % HR][c] = zc;
    st->h_zetat[i % HR][c] = ztc;
  }
}

template <class T> struct shift_of {
  static __device__ __forceinline__ T get(double re, double) { return T(re); }
};
template <class R> struct shift_of<cplx<R>> {
  static __device__ __forceinline__ cplx<R> get(double re, double im) { return cplx<R>((R)re, (R)im); }
};

// Op p at one row (Op = A or shift I - A).  `g(j)` returns the gathered vector entry.
template <class V, class T, class G>
__device__ __forceinline__ SpAcc<T> row_apply(const int* __restrict__ rp, const int* __restrict__ ci,
                                              const V* __restrict__ va, int row, G g) {
  SpAcc<T> acc;
  const int e0 = rp[row], e1 = rp[row + 1];
  for (int e = e0; e < e1; ++e) acc.add(va[e], g(ci[e]));
  return acc;
}

template <class A> __device__ __forceinline__ bool finite_acc(A v);
template <> __device__ __forceinline__ bool finite_acc<double>(double v) { return isfinite(v); }
template <> __device__ __forceinline__ bool finite_acc<zd>(zd v) { return isfinite(v.re) && isfinite(v.im); }

// ------------------------------------------------------------------------------------
// phase 1: dual SpMV with on-the-fly p update, projections
//
// The projections Ct^H z and C^H zt run over the contiguous 32 x LD slab of the row-major
// bases that belongs to a warp's 32 rows: element e = lane + 32 t of the slab is row e / LD,
// column e % LD, so loads are fully coalesced and every lane does useful work.  Because LD is a
// multiple of 4, lane `lane` only ever meets the P = LD / gcd(LD, 32) <= 7 columns
// (lane + 32 u) % LD, u < P, and keeps one accumulator per such column (slot u = t mod P).
// The block then folds the slots back to columns in a fixed order.
//
// Without a recycle space (LD = 0) q_i = z_i, so phase 2 has nothing left but the (pt, q)
// reduction; phase 1 does it and a plain iteration takes two launches.  Its rows are walked in
// the order of phase 2 (thread t: rows r0 + t + 256 j), so alpha is the same bit for bit either
// way (a request without recycle space in a batch with recycling requests runs both phases).
// ------------------------------------------------------------------------------------
constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }

template <int LD> struct Slab {
  static constexpr int G = cgcd(LD, 32);
  static constexpr int P = LD / G;
};

// Fold one side's per-lane slot accumulators red[warp][lane][u] (A type, shared memory) into
// per-block column sums out[c], c < LD; fixed order (deterministic).
template <class A, int LD>
__device__ void fold_slots(const A* red, A* wpart, int nwarps, A* out) {
  constexpr int P = Slab<LD>::P;
  // stage 1: item (c, w) sums over the lanes of warp w that hold column c
  for (int it = threadIdx.x; it < LD * nwarps; it += blockDim.x) {
    const int w = it % nwarps, c = it / nwarps;
    A sacc = A(0.0);
#pragma unroll
    for (int u = 0; u < P; ++u) {
      int l0 = (c - 32 * u) % LD;
      if (l0 < 0) l0 += LD;
      for (int l = l0; l < 32; l += LD) sacc += red[(w * 32 + l) * P + u];
    }
    wpart[c * nwarps + w] = sacc;
  }
  __syncthreads();
  // stage 2: column c sums over warps
  for (int c = threadIdx.x; c < LD; c += blockDim.x) {
    A sacc = A(0.0);
    for (int w = 0; w < nwarps; ++w) sacc += wpart[c * nwarps + w];
    out[c] = sacc;
  }
  __syncthreads();
}

template <class V, class T, int LD>
__device__ __forceinline__ void phase1_body(const OpArgs<V> op, const VecArgs<T> v, DevState* st,
                                            typename traits<T>::acc* part, Blk g) {
  typedef typename traits<T>::acc A;
  constexpr int NW = NTHREADS / 32;
  constexpr int LDA = LD > 0 ? LD : 4;
  constexpr int P = Slab<LDA>::P;
  __shared__ T zs[NW][32], zts[NW][32];
  __shared__ A red[LD > 0 ? NW * 32 * P : NW * 4];  // one side at a time
  __shared__ A wpart[LD > 0 ? LDA * NW : 1];
  __shared__ A tot[2 * LDA];
  pdl_wait();
  if (st->done) return;
  const int i = st->iter + 1;
  const T beta = from_zd<T>(st->beta), cbeta = conjg(beta);
  const zd rho_prev = st->rho;   // for alpha when this launch finishes it
  const int64_t so = (int64_t)((i - 1) % v.R) * v.ld;
  const T* __restrict__ r = v.ring + so;
  const T* __restrict__ rt = v.ringt + so;
  // (selects instead of indexing: the argument structs then stay in registers)
  const T* __restrict__ po = (i & 1) ? v.p[0] : v.p[1];
  const T* __restrict__ pto = (i & 1) ? v.pt[0] : v.pt[1];
  T* __restrict__ pn = (i & 1) ? v.p[1] : v.p[0];
  T* __restrict__ ptn = (i & 1) ? v.pt[1] : v.pt[0];
  const T sh = shift_of<T>::get(op.sh_re, op.sh_im), shc = conjg(sh);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T a1[P], a2[P];
#pragma unroll
  for (int u = 0; u < P; ++u) { a1[u] = T(0); a2[u] = T(0); }
  A pq = A(0.0), nq = A(0.0), npt = A(0.0);
  int r0, r1;
  block_rows(op.n, g, r0, r1);
  // Staged (one solve's launch, real types, when the launch gives the dynamic shared memory):
  // the block first forms p_i = r_{i-1} + beta p_{i-1} and pt_i for its rows and the op.bw rows
  // on either side -- every column its rows' nonzeros can reach -- in shared memory, and stores
  // its own rows once; the SpMV then gathers p from there instead of forming r_j + beta p_j again
  // for every nonzero.  The same expressions give the same values, so the results are unchanged.
  bool staged = false;
  int slo = 0;
  if constexpr (!traits<T>::cx) {
    if (op.stage_rows > 0 && op.bw > 0 && r1 > r0) {
      slo = r0 - op.bw > 0 ? r0 - op.bw : 0;
      const int shi = r1 + op.bw < op.n ? r1 + op.bw : op.n;
      staged = shi - slo <= op.stage_rows;   // block-uniform
      if (staged) {
        extern __shared__ __align__(16) unsigned char rb_phase1_dyn[];
        T* __restrict__ ps = reinterpret_cast<T*>(rb_phase1_dyn);
        T* __restrict__ pts = ps + op.stage_rows;
        for (int row = slo + (int)threadIdx.x; row < shi; row += NTHREADS) {
          const T prow = r[row] + beta * po[row];
          const T ptrow = rt[row] + cbeta * pto[row];
          ps[row - slo] = prow;
          pts[row - slo] = ptrow;
          if (row >= r0 && row < r1) {
            pn[row] = prow;
            ptn[row] = ptrow;
          }
        }
        __syncthreads();
        for (int base = r0 + warp * 32; base < r1; base += NTHREADS) {
          const int row = base + lane;
          T z = T(0), zt = T(0);
          if (row < r1) {
            SpAcc<T> za, zta;
            const int e0 = op.rp[row], e1 = op.rp[row + 1];
            if (op.shared) {
              for (int e = e0; e < e1; ++e) {
                const int j = op.ci[e];
                za.add(op.va[e], ps[j - slo]);
                zta.add(op.tva[e], pts[j - slo]);
              }
            } else {
              for (int e = e0; e < e1; ++e) {
                const int j = op.ci[e];
                za.add(op.va[e], ps[j - slo]);
              }
              const int f0 = op.trp[row], f1 = op.trp[row + 1];
              for (int e = f0; e < f1; ++e) {
                const int j = op.tci[e];
                zta.add(op.tva[e], pts[j - slo]);
              }
            }
            const T prow = ps[row - slo];
            const T ptrow = pts[row - slo];
            if (op.has_shift) { z = za.shifted(sh, prow); zt = zta.shifted(shc, ptrow); }
            else { z = za.value(); zt = zta.value(); }
            v.z[row] = z;
            v.zt[row] = zt;
            if (LD == 0) alpha_terms(pq, nq, npt, ptrow, z);
          }
          if (LD > 0) {
            zs[warp][lane] = z;
            zts[warp][lane] = zt;
            __syncwarp();
            const int nvalid = r1 - base < 32 ? r1 - base : 32;
            const T* __restrict__ ctb = v.Ct + (int64_t)base * LDA;
            const T* __restrict__ cb = v.C + (int64_t)base * LDA;
#pragma unroll
            for (int t = 0; t < LDA; ++t) {
              const int e = lane + 32 * t;
              const int rr = e / LDA;
              if (rr < nvalid) {
                a1[t % P] += cmul(ctb[e], zs[warp][rr]);
                a2[t % P] += cmul(cb[e], zts[warp][rr]);
              }
            }
            __syncwarp();
          }
        }
      }
    }
  }
  if (!staged) {
    for (int base = r0 + warp * 32; base < r1; base += NTHREADS) {
      const int row = base + lane;
      T z = T(0), zt = T(0);
      if (row < r1) {
        SpAcc<T> za, zta;
        const int e0 = op.rp[row], e1 = op.rp[row + 1];
        if (op.shared) {
          for (int e = e0; e < e1; ++e) {
            const int j = op.ci[e];
            za.add(op.va[e], r[j] + beta * po[j]);
            zta.add(op.tva[e], rt[j] + cbeta * pto[j]);
          }
        } else {
          for (int e = e0; e < e1; ++e) {
            const int j = op.ci[e];
            za.add(op.va[e], r[j] + beta * po[j]);
          }
          const int f0 = op.trp[row], f1 = op.trp[row + 1];
          for (int e = f0; e < f1; ++e) {
            const int j = op.tci[e];
            zta.add(op.tva[e], rt[j] + cbeta * pto[j]);
          }
        }
        const T prow = r[row] + beta * po[row];
        const T ptrow = rt[row] + cbeta * pto[row];
        pn[row] = prow;
        ptn[row] = ptrow;
        if (op.has_shift) { z = za.shifted(sh, prow); zt = zta.shifted(shc, ptrow); }
        else { z = za.value(); zt = zta.value(); }
        v.z[row] = z;
        v.zt[row] = zt;
        if (LD == 0) alpha_terms(pq, nq, npt, ptrow, z);
      }
      if (LD > 0) {
        zs[warp][lane] = z;
        zts[warp][lane] = zt;
        __syncwarp();
        const int nvalid = r1 - base < 32 ? r1 - base : 32;
        const T* __restrict__ ctb = v.Ct + (int64_t)base * LDA;
        const T* __restrict__ cb = v.C + (int64_t)base * LDA;
#pragma unroll
        for (int t = 0; t < LDA; ++t) {
          const int e = lane + 32 * t;
          const int rr = e / LDA;
          if (rr < nvalid) {
            a1[t % P] += cmul(ctb[e], zs[warp][rr]);
            a2[t % P] += cmul(cb[e], zts[warp][rr]);
          }
        }
        __syncwarp();
      }
    }
  }
  pdl_release();
  if (LD == 0) {
    block_sum3(pq, nq, npt, red, tot);
    if (!grid_reduce3(tot, red, part, st->gcnt, g)) return;
    finish_alpha(st, tot, i, 0, rho_prev);
    return;
  }
#pragma unroll
  for (int u = 0; u < P; ++u) red[(warp * 32 + lane) * P + u] = cvt<A>(a1[u]);
  __syncthreads();
  fold_slots<A, LDA>(red, wpart, NW, tot);          // Ct^H z  -> tot[0 .. LD)
#pragma unroll
  for (int u = 0; u < P; ++u) red[(warp * 32 + lane) * P + u] = cvt<A>(a2[u]);
  __syncthreads();
  fold_slots<A, LDA>(red, wpart, NW, tot + LDA);    // C^H zt  -> tot[LD .. 2 LD)
  if (!grid_reduce<A, 2 * LDA>(tot, part, st->gcnt, g)) return;
  const int k = st->kc;
  if (threadIdx.x < k) {
    const double d = st->Dc[threadIdx.x];
    st->zeta[threadIdx.x] = to_zd(tot[threadIdx.x] * (1.0 / d));
    st->zetat[threadIdx.x] = to_zd(tot[LDA + threadIdx.x] * (1.0 / d));
  }
}

// ------------------------------------------------------------------------------------
// phase 2: q = z - C zeta, qt = zt - Ct zetat, (pt, q) -> alpha
// ------------------------------------------------------------------------------------
template <class V, class T, int KT>
__device__ __forceinline__ void phase2_body(const OpArgs<V> op, const VecArgs<T> v, DevState* st,
                                            typename traits<T>::acc* part, Blk g) {
  typedef typename traits<T>::acc A;
  constexpr int KA = KT > 0 ? KT : 1;
  constexpr int NW = NTHREADS / 32;
  __shared__ A red[NW * 4];
  __shared__ A tot[3];
  __shared__ T ze[KA], zet[KA];   // zeta, zetat broadcast from shared memory (few registers)
  // per warp: an 8-column slice of C (or Ct) for its 32 rows, row stride 9 (conflict-free reads)
  __shared__ T stg[KT > 0 ? NW : 1][KT > 0 ? 32 * 9 : 1];
  pdl_wait();
  if (st->done) return;
  const int i = st->iter + 1;
  const int k = KT > 0 ? st->kc : 0;
  const zd rho_prev = st->rho;
  for (int c = threadIdx.x; c < KA; c += blockDim.x) {
    ze[c] = c < k ? from_zd<T>(st->zeta[c]) : T(0);
    zet[c] = c < k ? from_zd<T>(st->zetat[c]) : T(0);
  }
  __syncthreads();
  const T* __restrict__ pt = (i & 1) ? v.pt[1] : v.pt[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  A pq = A(0.0), nq = A(0.0), npt = A(0.0);
  int r0, r1;
  block_rows(op.n, g, r0, r1);
  // warp w takes the 32-row chunks r0 + 32 w + 256 j, so thread t sees rows r0 + t + 256 j:
  // the order in which phase 1 accumulates the same sums when it finishes alpha itself
  for (int base = r0 + warp * 32; base < r1; base += NTHREADS) {
    const int row = base + lane;
    const bool live = row < r1;
    T q = live ? v.z[row] : T(0), qt = live ? v.zt[row] : T(0);
    if (KT > 0) {
      // q = z - C zeta, qt = zt - Ct zetat, columns in ascending order.  A slice's 8 entries of
      // a row are 64 contiguous bytes, so each warp load reads 4 rows in whole sectors.
      const int nvalid = r1 - base < 32 ? r1 - base : 32;
      const int ldk = v.ldc;
      T* sg = stg[warp];
#pragma unroll 1
      for (int c0 = 0; c0 < KA; c0 += 8) {
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
          const T* __restrict__ src = side == 0 ? v.C : v.Ct;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = lane + 32 * u, rr = e >> 3, cc = c0 + (e & 7);
            sg[rr * 9 + (e & 7)] = (rr < nvalid && cc < ldk) ? src[(int64_t)(base + rr) * ldk + cc] : T(0);
          }
          __syncwarp();
          if (live) {
            T acc = side == 0 ? q : qt;
            const T* zz = side == 0 ? ze : zet;
#pragma unroll
            for (int cl = 0; cl < 8; ++cl)
              if (c0 + cl < k) acc -= sg[lane * 9 + cl] * zz[c0 + cl];
            if (side == 0) q = acc; else qt = acc;
          }
          __syncwarp();
        }
      }
      if (live) {
        v.z[row] = q;
        v.zt[row] = qt;
      }
    }
    if (live) alpha_terms(pq, nq, npt, pt[row], q);
  }
  pdl_release();
  block_sum3(pq, nq, npt, red, tot);
  if (!grid_reduce3(tot, red, part, st->gcnt, g)) return;
  finish_alpha(st, tot, i, k, rho_prev);
}

// ------------------------------------------------------------------------------------
// phase 3: x, r updates, rho, norms, stopping test, beta
// ------------------------------------------------------------------------------------
template <class V, class T>
__device__ __forceinline__ void phase3_body(const OpArgs<V> op, const VecArgs<T> v, DevState* st,
                                            typename traits<T>::acc* part, Blk g) {
  typedef typename traits<T>::acc A;
  __shared__ A red[(NTHREADS / 32) * 4];
  __shared__ A tot[3];
  pdl_wait();
  if (st->done) return;
  const int i = st->iter + 1;
  const T al = from_zd<T>(st->alpha), cal = conjg(al);
  // scalars of the finishing block, read up front (the kernel does not change them)
  const zd rho_prev = st->rho;
  const double tol = st->tol, bnorm = st->bnorm, btnorm = st->btnorm;
  const int max_itn = st->max_itn;
  const int64_t so = (int64_t)((i - 1) % v.R) * v.ld, sn = (int64_t)(i % v.R) * v.ld;
  const T* __restrict__ ro = v.ring + so;
  const T* __restrict__ rto = v.ringt + so;
  T* __restrict__ rn = v.ring + sn;
  T* __restrict__ rtn = v.ringt + sn;
  const T* __restrict__ p = (i & 1) ? v.p[1] : v.p[0];
  const T* __restrict__ pt = (i & 1) ? v.pt[1] : v.pt[0];
  A rho = A(0.0), n1 = A(0.0), n2 = A(0.0);
  int r0, r1;
  block_rows(op.n, g, r0, r1);
  T* __restrict__ x = v.x;
  T* __restrict__ xt = v.xt;
  const T* __restrict__ q = v.z;
  const T* __restrict__ qt = v.zt;
  int row = r0 + (int)threadIdx.x;
  // Real types take two rows a thread per step with all their loads issued first (the pointers
  // above do not alias), so more loads are in flight; the rows and the sums keep their order.
  constexpr int U = sizeof(T) <= 8 ? 2 : 1;
  if (U == 2) {
    for (; row + NTHREADS < r1; row += 2 * NTHREADS) {
      const int w = row + NTHREADS;
      const T x0 = x[row], x1 = x[w], p0 = p[row], p1 = p[w];
      const T xt0 = xt[row], xt1 = xt[w], pt0 = pt[row], pt1 = pt[w];
      const T ro0 = ro[row], ro1 = ro[w], q0 = q[row], q1 = q[w];
      const T rto0 = rto[row], rto1 = rto[w], qt0 = qt[row], qt1 = qt[w];
      x[row] = x0 + al * p0;
      xt[row] = xt0 + cal * pt0;
      const T a0 = ro0 - al * q0;
      const T b0 = rto0 - cal * qt0;
      rn[row] = a0;
      rtn[row] = b0;
      rho += cmul(cvt<A>(b0), cvt<A>(a0));
      n1 += A((double)abs2(a0));
      n2 += A((double)abs2(b0));
      x[w] = x1 + al * p1;
      xt[w] = xt1 + cal * pt1;
      const T a1 = ro1 - al * q1;
      const T b1 = rto1 - cal * qt1;
      rn[w] = a1;
      rtn[w] = b1;
      rho += cmul(cvt<A>(b1), cvt<A>(a1));
      n1 += A((double)abs2(a1));
      n2 += A((double)abs2(b1));
    }
  }
  for (; row < r1; row += NTHREADS) {
    x[row] = x[row] + al * p[row];
    xt[row] = xt[row] + cal * pt[row];
    const T a = ro[row] - al * q[row];
    const T b = rto[row] - cal * qt[row];
    rn[row] = a;
    rtn[row] = b;
    rho += cmul(cvt<A>(b), cvt<A>(a));
    n1 += A((double)abs2(a));
    n2 += A((double)abs2(b));
  }
  pdl_release();
  block_sum3(rho, n1, n2, red, tot);
  if (!grid_reduce3(tot, red, part, st->gcnt, g)) return;
  if (threadIdx.x == 0) {
    const zd RHO = to_zd(tot[0]);
    const double rr = sqrt(real_of(tot[1])), rtr = sqrt(real_of(tot[2]));
    const zd beta = RHO * crcp(rho_prev);
    st->h_rnorm[i % HR] = rr;
    st->h_rho[i % HR] = RHO;
    st->h_beta[i % HR] = beta;
    st->rnorm = rr;
    st->rtnorm = rtr;
    st->iter = i;
    const bool conv = rr <= tol * bnorm && (btnorm == 0.0 || rtr <= tol * btnorm);
    if (!isfinite(rr) || !isfinite(rtr) || !isfinite(RHO.re) || !isfinite(RHO.im)) st->done = DONE_NONFINITE;
    else if (conv) st->done = DONE_CONVERGED;
    else if (abs2(RHO) <= (BREAKDOWN_EPS * rr * rtr) * (BREAKDOWN_EPS * rr * rtr)) st->done = DONE_BREAK_RHO;
    else if (i >= max_itn) st->done = DONE_MAXIT;
    st->rho = RHO;
    st->beta = beta;
  }
}


// Single-solve kernels and their batched forms (one launch for every request of a batch).
template <class V, class T>
__device__ __forceinline__ int batch_slot(const BatchArgs<V, T>* ba) {
  int r = 0;
  while (r + 1 < ba->nreq && (int)blockIdx.x >= ba->start[r + 1]) ++r;
  return r;
}
// MINB resident blocks per SM: the unrolled slab projection of phase 1 otherwise takes 128
// registers a thread and halves the warps that hide the gather latency.  Three blocks per SM is
// the default grid's one wave without recycling (3 x SMs blocks; with recycling the default is
// 2 x SMs, leaving room for the concurrent refresh); phase 2's staged slices need that many
// registers to stay out of local memory.
#define RB_PHASE_KERNELS(NAME, BODY, MINB, TPARAMS, TARGS)                                               \
  template <TPARAMS>                                                                                    \
  __global__ void __launch_bounds__(NTHREADS, MINB) NAME(OpArgs<V> op, VecArgs<T> v, DevState* st,     \
                                                         typename traits<T>::acc* part) {              \
    BODY<TARGS>(op, v, st, part, Blk{(int)blockIdx.x, (int)gridDim.x});                                 \
  }                                                                                                     \
  template <TPARAMS>                                                                                    \
  __global__ void __launch_bounds__(NTHREADS, MINB) NAME##_b(const BatchArgs<V, T>* __restrict__ ba) { \
    const int r = batch_slot(ba);                                                                       \
    OpArgs<V> op = ba->op[r];                                                                           \
    op.stage_rows = 0;   /* batched launches give no dynamic shared memory */                          \
    const VecArgs<T> v = ba->v[r];                                                                      \
    BODY<TARGS>(op, v, ba->st[r], reinterpret_cast<typename traits<T>::acc*>(ba->part[r]),             \
                Blk{(int)blockIdx.x - ba->start[r], ba->start[r + 1] - ba->start[r]});                  \
  }
#define RB_COMMA ,
RB_PHASE_KERNELS(k_phase1, phase1_body, 3, class V RB_COMMA class T RB_COMMA int LD, V RB_COMMA T RB_COMMA LD)
RB_PHASE_KERNELS(k_phase2, phase2_body, 3, class V RB_COMMA class T RB_COMMA int KT, V RB_COMMA T RB_COMMA KT)
RB_PHASE_KERNELS(k_phase3, phase3_body, 3, class V RB_COMMA class T, V RB_COMMA T)
#undef RB_COMMA
#undef RB_PHASE_KERNELS

// ------------------------------------------------------------------------------------
// initial projection, eq. (minusXR): r_{-1} = b - Op x_{-1}, coef = D_c^{-1} Ct^H r_{-1},
// x_0 = x_{-1} + U coef, r_0 = r_{-1} - C coef (and the dual with Ut, C, Ct swapped).
// ------------------------------------------------------------------------------------
template <class V, class T, int KT>
__global__ void __launch_bounds__(NTHREADS) k_init_a(OpArgs<V> op, VecArgs<T> v, DevState* st,
                                                     typename traits<T>::acc* part, int dual_only) {
  typedef typename traits<T>::acc A;
  constexpr int KA = KT > 0 ? KT : 1;
  constexpr int CNT = 2 * KA + 2;
  __shared__ A red[(NTHREADS / 32) * CNT];
  __shared__ A tot[CNT];
  T* __restrict__ r = v.ring;   // slot 0 holds r_{-1}, then r_0
  T* __restrict__ rt = v.ringt;
  const int k = KT > 0 ? st->kc : 0;
  const T sh = shift_of<T>::get(op.sh_re, op.sh_im), shc = conjg(sh);
  T a1[KA], a2[KA];
  A nb = A(0.0), nbt = A(0.0);
#pragma unroll
  for (int c = 0; c < KA; ++c) { a1[c] = T(0); a2[c] = T(0); }
  const T* __restrict__ x = v.x;
  const T* __restrict__ xt = v.xt;
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < op.n; row += stride) {
    T res = T(0), rest = T(0);
    if (!dual_only) {
      const SpAcc<T> aa = row_apply<V, T>(op.rp, op.ci, op.va, row, [&](int j) { return x[j]; });
      const T ax = op.has_shift ? aa.shifted(sh, x[row]) : aa.value();
      res = v.b[row] - ax;
      r[row] = res;
      nb += A((double)abs2(v.b[row]));
    }
    const SpAcc<T> ta = row_apply<V, T>(op.trp, op.tci, op.tva, row, [&](int j) { return xt[j]; });
    const T atx = op.has_shift ? ta.shifted(shc, xt[row]) : ta.value();
    rest = v.bt[row] - atx;
    rt[row] = rest;
    nbt += A((double)abs2(v.bt[row]));
    if (KT > 0) {
      const T* __restrict__ crow = v.C + (int64_t)row * v.ldc;
      const T* __restrict__ ctrow = v.Ct + (int64_t)row * v.ldc;
#pragma unroll
      for (int c = 0; c < KA; ++c)
        if (c < k) { a1[c] += cmul(ctrow[c], res); a2[c] += cmul(crow[c], rest); }
    }
  }
  A vals[CNT];
#pragma unroll
  for (int c = 0; c < KA; ++c) { vals[c] = cvt<A>(a1[c]); vals[KA + c] = cvt<A>(a2[c]); }
  vals[2 * KA] = nb;
  vals[2 * KA + 1] = nbt;
  write_partials(vals, CNT, red, part, (int)blockIdx.x);
  if (!arrive_last(&st->cnt[3], (int)gridDim.x)) return;
  reduce_cols(part, gridDim.x, CNT, tot);
  if (threadIdx.x < k) {
    const double d = st->Dc[threadIdx.x];
    if (!dual_only) st->coef[threadIdx.x] = to_zd(tot[threadIdx.x] * (1.0 / d));
    st->coeft[threadIdx.x] = to_zd(tot[KA + threadIdx.x] * (1.0 / d));
  }
  if (threadIdx.x == 0) {
    if (!dual_only) st->bnorm = sqrt(real_of(tot[2 * KA]));
    st->btnorm = sqrt(real_of(tot[2 * KA + 1]));
  }
}

template <class V, class T, int KT>
__global__ void __launch_bounds__(NTHREADS) k_init_b(OpArgs<V> op, VecArgs<T> v, DevState* st,
                                                     typename traits<T>::acc* part, int dual_only) {
  typedef typename traits<T>::acc A;
  constexpr int KA = KT > 0 ? KT : 1;
  __shared__ A red[(NTHREADS / 32) * 3];
  __shared__ A tot[3];
  const int k = KT > 0 ? st->kc : 0;
  T cf[KA], cft[KA];
#pragma unroll
  for (int c = 0; c < KA; ++c) {
    cf[c] = c < k ? from_zd<T>(st->coef[c]) : T(0);
    cft[c] = c < k ? from_zd<T>(st->coeft[c]) : T(0);
  }
  T* __restrict__ r = v.ring;
  T* __restrict__ rt = v.ringt;
  A rho = A(0.0), n1 = A(0.0), n2 = A(0.0);
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < op.n; row += stride) {
    T a = r[row], b = rt[row];
    if (KT > 0) {
      const int64_t o = (int64_t)row * v.ldk, oc = (int64_t)row * v.ldc;
      T dx = T(0), dr = T(0), dxt = T(0), drt = T(0);
#pragma unroll
      for (int c = 0; c < KA; ++c)
        if (c < k) {
          if (!dual_only) { dx += v.U[o + c] * cf[c]; dr += v.C[oc + c] * cf[c]; }
          dxt += v.Ut[o + c] * cft[c];
          drt += v.Ct[oc + c] * cft[c];
        }
      if (!dual_only) { v.x[row] = v.x[row] + dx; a = a - dr; r[row] = a; }
      v.xt[row] = v.xt[row] + dxt;
      b = b - drt;
      rt[row] = b;
    }
    v.p[0][row] = T(0);
    v.pt[0][row] = T(0);
    rho += cmul(cvt<A>(b), cvt<A>(a));
    n1 += A((double)abs2(a));
    n2 += A((double)abs2(b));
  }
  A vals[3] = {rho, n1, n2};
  write_partials(vals, 3, red, part, (int)blockIdx.x);
  if (!arrive_last(&st->cnt[4], (int)gridDim.x)) return;
  reduce_cols(part, gridDim.x, 3, tot);
  if (threadIdx.x < KMAX) { st->zeta_c[threadIdx.x] = zd(); st->zetat_c[threadIdx.x] = zd(); }
  if (threadIdx.x == 0) {
    const zd RHO = to_zd(tot[0]);
    const double rr = sqrt(real_of(tot[1])), rtr = sqrt(real_of(tot[2]));
    st->rho = RHO;
    st->beta = zd();
    st->iter = 0;
    st->rnorm = rr;
    st->rtnorm = rtr;
    st->h_rho[0] = RHO;
    st->h_rnorm[0] = rr;
    st->h_beta[0] = zd();
    st->h_alpha[0] = zd();
    for (int c = 0; c < KMAX; ++c) { st->h_zeta[0][c] = zd(); st->h_zetat[0][c] = zd(); }
    const bool conv = rr <= st->tol * st->bnorm && (st->btnorm == 0.0 || rtr <= st->tol * st->btnorm);
    st->restart = (absval(RHO) <= BREAKDOWN_EPS * rr * rtr) && !conv;
    st->done = conv ? DONE_CONVERGED : RUNNING;
    if (!isfinite(rr) || !isfinite(rtr)) st->done = DONE_NONFINITE;
  }
}

// ------------------------------------------------------------------------------------
// step 7 (x -= U zeta_c, xt -= Ut zetat_c) and the FP64 true residual
// ------------------------------------------------------------------------------------
template <class T, int KT>
__global__ void __launch_bounds__(NTHREADS) k_fin_a(int n, VecArgs<T> v, DevState* st) {
  constexpr int KA = KT > 0 ? KT : 1;
  const int k = st->kc;
  T zc[KA], ztc[KA];
#pragma unroll
  for (int c = 0; c < KA; ++c) {
    zc[c] = c < k ? from_zd<T>(st->zeta_c[c]) : T(0);
    ztc[c] = c < k ? from_zd<T>(st->zetat_c[c]) : T(0);
  }
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += stride) {
    const int64_t o = (int64_t)row * v.ldk;
    T dx = T(0), dxt = T(0);
#pragma unroll
    for (int c = 0; c < KA; ++c)
      if (c < k) { dx += v.U[o + c] * zc[c]; dxt += v.Ut[o + c] * ztc[c]; }
    v.x[row] = v.x[row] - dx;
    v.xt[row] = v.xt[row] - dxt;
  }
}

template <class V, class T>
__global__ void __launch_bounds__(NTHREADS) k_fin_b(OpArgs<V> op, VecArgs<T> v, DevState* st,
                                                    typename traits<T>::acc* part) {
  typedef typename traits<T>::acc A;
  __shared__ A red[(NTHREADS / 32) * 2];
  __shared__ A tot[2];
  const T sh = shift_of<T>::get(op.sh_re, op.sh_im), shc = conjg(sh);
  const T* __restrict__ x = v.x;
  const T* __restrict__ xt = v.xt;
  A n1 = A(0.0), n2 = A(0.0);
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < op.n; row += stride) {
    const SpAcc<T> aa = row_apply<V, T>(op.rp, op.ci, op.va, row, [&](int j) { return x[j]; });
    const T ax = op.has_shift ? aa.shifted(sh, x[row]) : aa.value();
    const SpAcc<T> ta = row_apply<V, T>(op.trp, op.tci, op.tva, row, [&](int j) { return xt[j]; });
    const T atx = op.has_shift ? ta.shifted(shc, xt[row]) : ta.value();
    n1 += A((double)abs2(v.b[row] - ax));
    n2 += A((double)abs2(v.bt[row] - atx));
  }
  A vals[2] = {n1, n2};
  write_partials(vals, 2, red, part, (int)blockIdx.x);
  if (!arrive_last(&st->cnt[5], (int)gridDim.x)) return;
  reduce_cols(part, gridDim.x, 2, tot);
  if (threadIdx.x == 0) {
    st->true_rnorm = sqrt(real_of(tot[0]));
    st->true_rtnorm = sqrt(real_of(tot[1]));
  }
}

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) restart vector in [-1, 1): element e uses counter
// (e lo, e hi, 0, 0) and key (seed lo, seed hi); top 53 bits of (w1:w0) [and (w3:w2)].
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}
__device__ __forceinline__ double u53(uint32_t lo, uint32_t hi) {
  const uint64_t w = ((uint64_t)hi << 32) | lo;
  return 2.0 * ((double)(w >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}
template <class T> struct philox_store;
template <> struct philox_store<double> {
  static __device__ void put(double* o, const uint32_t c[4]) { *o = u53(c[0], c[1]); }
};
template <> struct philox_store<float> {
  static __device__ void put(float* o, const uint32_t c[4]) { *o = (float)u53(c[0], c[1]); }
};
template <class R> struct philox_store<cplx<R>> {
  static __device__ void put(cplx<R>* o, const uint32_t c[4]) { *o = cplx<R>((R)u53(c[0], c[1]), (R)u53(c[2], c[3])); }
};
template <class T>
__global__ void k_philox(T* out, int64_t n, uint64_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)(e & 0xffffffffu), (uint32_t)(e >> 32), 0u, 0u};
    philox10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    philox_store<T>::put(out + e, c);
  }
}

// ------------------------------------------------------------------------------------
// CSR validation and A^H construction
// ------------------------------------------------------------------------------------
__global__ void k_validate(int n, int64_t nnz, const int* rp, const int* ci, int* flag) {
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += stride) {
    const int e0 = rp[row], e1 = rp[row + 1];
    if (row == 0 && e0 != 0) atomicOr(flag, 1);
    if (row == n - 1 && (int64_t)e1 != nnz) atomicOr(flag, 2);
    if (e1 < e0 || e0 < 0 || (int64_t)e1 > nnz) { atomicOr(flag, 4); continue; }
    int prev = -1;
    for (int e = e0; e < e1; ++e) {
      const int j = ci[e];
      if (j < 0 || j >= n) atomicOr(flag, 8);
      if (j <= prev) atomicOr(flag, 16);
      prev = j;
    }
  }
}

// bandwidth: max |j - i| over the nonzeros (columns sorted, so a row's first and last decide)
__global__ void k_bandwidth(int n, const int* rp, const int* ci, int* bw) {
  int m = 0;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    const int e0 = rp[row], e1 = rp[row + 1];
    if (e1 > e0) {
      const int lo = row - ci[e0], hi = ci[e1 - 1] - row;
      m = max(m, max(lo, hi));
    }
  }
  if (m > 0) atomicMax(bw, m);
}

RB_HD double conjv(double a) { return a; }
RB_HD float conjv(float a) { return a; }
template <class R> RB_HD cplx<R> conjv(cplx<R> a) { return conjg(a); }

// Structurally symmetric pattern: the A^H entry at (i, j) is conj(A(j, i)), found by binary
// search in row j.  flag |= 1 when some (j, i) is missing.
template <class V>
__global__ void k_adj_shared(int n, const int* rp, const int* ci, const V* va, V* tva, int* flag) {
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += stride) {
    const int e0 = rp[row], e1 = rp[row + 1];
    for (int e = e0; e < e1; ++e) {
      const int j = ci[e];
      int lo = rp[j], hi = rp[j + 1] - 1, f = -1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1, cm = ci[mid];
        if (cm == row) { f = mid; break; }
        if (cm < row) lo = mid + 1; else hi = mid - 1;
      }
      if (f < 0) { atomicOr(flag, 1); tva[e] = V(0); }
      else tva[e] = conjv(va[f]);
    }
  }
}

__global__ void k_count_cols(int n, const int* rp, const int* ci, int* cnt) {
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += stride)
    for (int e = rp[row]; e < rp[row + 1]; ++e) atomicAdd(cnt + ci[e], 1);
}

// exclusive scan in place over a[0..m) by one block (setup only)
__global__ void k_scan_one_block(int* a, int m) {
  __shared__ int sums[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int chunk = (m + T - 1) / T;
  const int b = t * chunk, e = min(m, b + chunk);
  int s = 0;
  for (int i = b; i < e; ++i) s += a[i];
  sums[t] = s;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int i = 0; i < T; ++i) { const int v = sums[i]; sums[i] = acc; acc += v; }
  }
  __syncthreads();
  int acc = sums[t];
  for (int i = b; i < e; ++i) { const int v = a[i]; a[i] = acc; acc += v; }
}

template <class V>
__global__ void k_scatter_adj(int n, const int* rp, const int* ci, const V* va, const int* trp, int* cursor,
                              int* tci, V* tva) {
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += stride)
    for (int e = rp[row]; e < rp[row + 1]; ++e) {
      const int j = ci[e];
      const int pos = trp[j] + atomicAdd(cursor + j, 1);
      tci[pos] = row;
      tva[pos] = conjv(va[e]);
    }
}

template <class V>
__global__ void k_sort_rows(int n, const int* trp, int* tci, V* tva) {
  const int stride = gridDim.x * blockDim.x;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += stride) {
    const int e0 = trp[row], e1 = trp[row + 1];
    for (int a = e0 + 1; a < e1; ++a) {
      const int c = tci[a];
      const V v = tva[a];
      int b = a - 1;
      while (b >= e0 && tci[b] > c) { tci[b + 1] = tci[b]; tva[b + 1] = tva[b]; --b; }
      tci[b + 1] = c;
      tva[b + 1] = v;
    }
  }
}

// dst row r = src row r's first kc entries, zero-padded to ldd (the compact projection bases)
template <class T>
__global__ void k_pack_cols(const T* __restrict__ src, int lds, T* __restrict__ dst, int ldd, int kc, int64_t n) {
  const int64_t total = n * ldd;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ldd;
    const int c = (int)(e - r * ldd);
    dst[e] = c < kc ? src[r * lds + c] : T(0);
  }
}
template <class T>
void launch_pack_cols(const T* src, int lds, T* dst, int ldd, int kc, int64_t n, cudaStream_t s) {
  k_pack_cols<T><<<1024, 256, 0, s>>>(src, lds, dst, ldd, kc, n);
}
template void launch_pack_cols<double>(const double*, int, double*, int, int, int64_t, cudaStream_t);
template void launch_pack_cols<float>(const float*, int, float*, int, int, int64_t, cudaStream_t);
template void launch_pack_cols<zd>(const zd*, int, zd*, int, int, int64_t, cudaStream_t);
template void launch_pack_cols<cplx<float>>(const cplx<float>*, int, cplx<float>*, int, int, int64_t, cudaStream_t);

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
#define RB_KT_DISPATCH(kt, CALL) \
  switch (kt) {                  \
    case 0: CALL(0); break;      \
    case 8: CALL(8); break;      \
    case 16: CALL(16); break;    \
    case 24: CALL(24); break;    \
    default: CALL(32); break;    \
  }

// Iteration-phase launches use programmatic stream serialization (pdl_wait / pdl_release in
// the kernels), unless RBICG_NO_PDL is set in the environment.
static bool pdl_enabled() {
  static const bool on = getenv("RBICG_NO_PDL") == nullptr;
  return on;
}
template <class... KArgs, class... Args>
static void launch_phase_kernel(void (*k)(KArgs...), int grid, cudaStream_t s, size_t dyn, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, args...);
}

// Phase-1 staging (see phase1_body): the dynamic shared memory a launch may give, from the SM's
// shared memory shared by the blocks that the grid puts on one SM and each instantiation's own
// static shared memory.  prepare_phase1() reads the static sizes and raises the kernels' dynamic
// limit once per (V, T), outside any stream capture; launches before it stage nothing.
constexpr int PHASE1_LDS[9] = {0, 4, 8, 12, 16, 20, 24, 28, 32};
template <class V, class T>
struct Phase1Smem {
  static bool ready;
  static int static_bytes[9];
  static int sm_bytes;   // shared memory per SM usable by blocks
  static int sms;
};
template <class V, class T> bool Phase1Smem<V, T>::ready = false;
template <class V, class T> int Phase1Smem<V, T>::static_bytes[9] = {};
template <class V, class T> int Phase1Smem<V, T>::sm_bytes = 0;
template <class V, class T> int Phase1Smem<V, T>::sms = 1;

template <class V, class T, int L>
static void prepare_one(int i, int max_dyn) {
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, k_phase1<V, T, L>);
  Phase1Smem<V, T>::static_bytes[i] = (int)fa.sharedSizeBytes;
  cudaFuncSetAttribute(k_phase1<V, T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       max_dyn - (int)fa.sharedSizeBytes);
}

template <class V, class T>
void prepare_phase1() {
  if (Phase1Smem<V, T>::ready || traits<T>::cx) return;
  int dev = 0, per_block = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&Phase1Smem<V, T>::sms, cudaDevAttrMultiProcessorCount, dev);
  Phase1Smem<V, T>::sm_bytes = per_sm;
  prepare_one<V, T, 0>(0, per_block);
  prepare_one<V, T, 4>(1, per_block);
  prepare_one<V, T, 8>(2, per_block);
  prepare_one<V, T, 12>(3, per_block);
  prepare_one<V, T, 16>(4, per_block);
  prepare_one<V, T, 20>(5, per_block);
  prepare_one<V, T, 24>(6, per_block);
  prepare_one<V, T, 28>(7, per_block);
  prepare_one<V, T, 32>(8, per_block);
  Phase1Smem<V, T>::ready = cudaGetLastError() == cudaSuccess;
}

// rows per side a launch stages: the largest block's rows plus bw on either side, if that fits
// beside the static shared memory of the blocks one SM holds (1 KB reserved per block); else 0
template <class V, class T>
static int phase1_stage_rows(const OpArgs<V>& op, int grid, int li) {
  if (traits<T>::cx || !Phase1Smem<V, T>::ready || op.bw <= 0 || op.n <= 0 || grid <= 0) return 0;
  static const bool off = getenv("RBICG_NO_STAGE") != nullptr;   // for tests and measurements
  if (off) return 0;
  const int64_t nch = ((int64_t)op.n + 31) / 32;
  const int64_t rows = std::min<int64_t>(op.n, (nch + grid - 1) / grid * 32 + 2 * (int64_t)op.bw);
  const int per_sm_blocks = (grid + Phase1Smem<V, T>::sms - 1) / Phase1Smem<V, T>::sms;
  const int64_t budget = Phase1Smem<V, T>::sm_bytes / std::max(1, per_sm_blocks) - 1024 -
                         Phase1Smem<V, T>::static_bytes[li];
  return rows * 2 * (int64_t)sizeof(T) <= budget ? (int)rows : 0;
}

template <class V, class T>
void launch_phase1(const OpArgs<V>& op_in, const VecArgs<T>& v, DevState* st, void* part, int kt, int grid,
                   cudaStream_t s) {
  typedef typename traits<T>::acc A;
  // kt == 0: no recycle space (no projection); otherwise dispatch on the bases' row stride
  const int ld = kt == 0 ? 0 : v.ldc;
  int li = 0;
  while (li < 8 && PHASE1_LDS[li] < ld) ++li;
  OpArgs<V> op = op_in;
  op.stage_rows = phase1_stage_rows<V, T>(op, grid, li);
  const size_t dyn = (size_t)op.stage_rows * 2 * sizeof(T);
#define RB_CALL(L) launch_phase_kernel(k_phase1<V, T, L>, grid, s, dyn, op, v, st, (A*)part)
  switch (ld) {
    case 0: RB_CALL(0); break;
    case 4: RB_CALL(4); break;
    case 8: RB_CALL(8); break;
    case 12: RB_CALL(12); break;
    case 16: RB_CALL(16); break;
    case 20: RB_CALL(20); break;
    case 24: RB_CALL(24); break;
    case 28: RB_CALL(28); break;
    default: RB_CALL(32); break;
  }
#undef RB_CALL
}
template <class V, class T>
void launch_phase2(const OpArgs<V>& op, const VecArgs<T>& v, DevState* st, void* part, int kt, int grid,
                   cudaStream_t s) {
  typedef typename traits<T>::acc A;
#define RB_CALL(K) launch_phase_kernel(k_phase2<V, T, K>, grid, s, (size_t)0, op, v, st, (A*)part)
  RB_KT_DISPATCH(kt, RB_CALL)
#undef RB_CALL
}
template <class V, class T>
void launch_phase3(const OpArgs<V>& op, const VecArgs<T>& v, DevState* st, void* part, int grid,
                   cudaStream_t s) {
  typedef typename traits<T>::acc A;
  launch_phase_kernel(k_phase3<V, T>, grid, s, (size_t)0, op, v, st, (A*)part);
}
template <class V, class T>
void launch_phase1_batch(const BatchArgs<V, T>* ba, int blocks, int ld, cudaStream_t s) {
#define RB_CALL(L) launch_phase_kernel(k_phase1_b<V, T, L>, blocks, s, (size_t)0, ba)
  switch (ld) {
    case 0: RB_CALL(0); break;
    case 4: RB_CALL(4); break;
    case 8: RB_CALL(8); break;
    case 12: RB_CALL(12); break;
    case 16: RB_CALL(16); break;
    case 20: RB_CALL(20); break;
    case 24: RB_CALL(24); break;
    case 28: RB_CALL(28); break;
    default: RB_CALL(32); break;
  }
#undef RB_CALL
}
template <class V, class T>
void launch_phase2_batch(const BatchArgs<V, T>* ba, int blocks, int kt, cudaStream_t s) {
#define RB_CALL(K) launch_phase_kernel(k_phase2_b<V, T, K>, blocks, s, (size_t)0, ba)
  RB_KT_DISPATCH(kt, RB_CALL)
#undef RB_CALL
}
template <class V, class T>
void launch_phase3_batch(const BatchArgs<V, T>* ba, int blocks, cudaStream_t s) {
  launch_phase_kernel(k_phase3_b<V, T>, blocks, s, (size_t)0, ba);
}
template <class V, class T>
void launch_init(const OpArgs<V>& op, const VecArgs<T>& v, DevState* st, void* part, int kt, int grid,
                 int dual_only, cudaStream_t s) {
  typedef typename traits<T>::acc A;
#define RB_CALL(K) k_init_a<V, T, K><<<grid, NTHREADS, 0, s>>>(op, v, st, (A*)part, dual_only)
  RB_KT_DISPATCH(kt, RB_CALL)
#undef RB_CALL
#define RB_CALL(K) k_init_b<V, T, K><<<grid, NTHREADS, 0, s>>>(op, v, st, (A*)part, dual_only)
  RB_KT_DISPATCH(kt, RB_CALL)
#undef RB_CALL
}
template <class V, class T>
void launch_finish(const OpArgs<V>& op, const VecArgs<T>& v, DevState* st, void* part, int kt, int grid,
                   cudaStream_t s) {
  typedef typename traits<T>::acc A;
#define RB_CALL(K) k_fin_a<T, K><<<grid, NTHREADS, 0, s>>>(op.n, v, st)
  RB_KT_DISPATCH(kt, RB_CALL)
#undef RB_CALL
  k_fin_b<V, T><<<grid, NTHREADS, 0, s>>>(op, v, st, (A*)part);
}
template <class T>
void launch_finish_a(const VecArgs<T>& v, DevState* st, int kt, int grid, cudaStream_t s) {
#define RB_CALL(K) k_fin_a<T, K><<<grid, NTHREADS, 0, s>>>((int)v.n, v, st)
  RB_KT_DISPATCH(kt, RB_CALL)
#undef RB_CALL
}
template <class T>
void launch_philox(T* out, int64_t n, uint64_t seed, cudaStream_t s) {
  k_philox<T><<<256, 256, 0, s>>>(out, n, seed);
}

int validate_csr(int n, int64_t nnz, const int* rp, const int* ci, int* flag_dev, cudaStream_t s) {
  cudaMemsetAsync(flag_dev, 0, sizeof(int), s);
  k_validate<<<std::max(1, std::min((n + 255) / 256, 1024)), 256, 0, s>>>(n, nnz, rp, ci, flag_dev);
  return (int)cudaGetLastError();
}

int csr_bandwidth(int n, const int* rp, const int* ci, int* flag_dev, cudaStream_t s, int* bw) {
  cudaMemsetAsync(flag_dev, 0, sizeof(int), s);
  k_bandwidth<<<std::max(1, std::min((n + 255) / 256, 1024)), 256, 0, s>>>(n, rp, ci, flag_dev);
  cudaMemcpyAsync(bw, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  return (int)cudaStreamSynchronize(s);
}

template <class V>
int build_adjoint(int n, const int* rp, const int* ci, const V* va, int** trp, int** tci, V** tva, int* shared,
                  int* flag_dev, cudaStream_t s) {
  // *tva must hold nnz values; *trp / *tci are allocated here only for unsymmetric patterns.
  const int grid = std::max(1, std::min((n + 255) / 256, 2048));
  cudaMemsetAsync(flag_dev, 0, sizeof(int), s);
  k_adj_shared<V><<<grid, 256, 0, s>>>(n, rp, ci, va, *tva, flag_dev);
  int flag = 0;
  cudaMemcpyAsync(&flag, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return (int)e;
  if (flag == 0) {
    *shared = 1;
    *trp = const_cast<int*>(rp);
    *tci = const_cast<int*>(ci);
    return 0;
  }
  *shared = 0;
  int nnz = 0;
  cudaMemcpyAsync(&nnz, rp + n, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  int* cur = nullptr;
  if ((e = cudaMalloc(trp, sizeof(int) * (n + 1))) != cudaSuccess) return (int)e;
  if ((e = cudaMalloc(tci, sizeof(int) * std::max(1, nnz))) != cudaSuccess) return (int)e;
  if ((e = cudaMalloc(&cur, sizeof(int) * (n + 1))) != cudaSuccess) return (int)e;
  cudaMemsetAsync(*trp, 0, sizeof(int) * (n + 1), s);
  cudaMemsetAsync(cur, 0, sizeof(int) * (n + 1), s);
  k_count_cols<<<grid, 256, 0, s>>>(n, rp, ci, *trp);   // trp[c] = entries in column c
  k_scan_one_block<<<1, 1024, 0, s>>>(*trp, n + 1);     // exclusive scan -> row starts of A^H
  k_scatter_adj<V><<<grid, 256, 0, s>>>(n, rp, ci, va, *trp, cur, *tci, *tva);
  k_sort_rows<V><<<grid, 256, 0, s>>>(n, *trp, *tci, *tva);
  e = cudaStreamSynchronize(s);
  cudaFree(cur);
  return (int)e;
}

// ------------------------------------------------------------------------------------
// explicit instantiations
// ------------------------------------------------------------------------------------
#define RB_INST_VT(V, T)                                                                                  \
  template void prepare_phase1<V, T>();                                                                     \
  template void launch_phase1<V, T>(const OpArgs<V>&, const VecArgs<T>&, DevState*, void*, int, int,       \
                                    cudaStream_t);                                                         \
  template void launch_phase2<V, T>(const OpArgs<V>&, const VecArgs<T>&, DevState*, void*, int, int,       \
                                    cudaStream_t);                                                         \
  template void launch_phase1_batch<V, T>(const BatchArgs<V, T>*, int, int, cudaStream_t);                 \
  template void launch_phase2_batch<V, T>(const BatchArgs<V, T>*, int, int, cudaStream_t);                 \
  template void launch_phase3_batch<V, T>(const BatchArgs<V, T>*, int, cudaStream_t);                      \
  template void launch_phase3<V, T>(const OpArgs<V>&, const VecArgs<T>&, DevState*, void*, int,            \
                                    cudaStream_t);                                                         \
  template void launch_init<V, T>(const OpArgs<V>&, const VecArgs<T>&, DevState*, void*, int, int, int,    \
                                  cudaStream_t);                                                           \
  template void launch_finish<V, T>(const OpArgs<V>&, const VecArgs<T>&, DevState*, void*, int, int,       \
                                    cudaStream_t);

RB_INST_VT(double, double)
RB_INST_VT(float, float)
RB_INST_VT(double, cplx<double>)
RB_INST_VT(cplx<double>, cplx<double>)
RB_INST_VT(float, cplx<float>)
RB_INST_VT(cplx<float>, cplx<float>)

template void launch_finish_a<double>(const VecArgs<double>&, DevState*, int, int, cudaStream_t);
template void launch_finish_a<float>(const VecArgs<float>&, DevState*, int, int, cudaStream_t);
template void launch_finish_a<cplx<double>>(const VecArgs<cplx<double>>&, DevState*, int, int, cudaStream_t);
template void launch_finish_a<cplx<float>>(const VecArgs<cplx<float>>&, DevState*, int, int, cudaStream_t);
template void launch_philox<double>(double*, int64_t, uint64_t, cudaStream_t);
template void launch_philox<float>(float*, int64_t, uint64_t, cudaStream_t);
template void launch_philox<cplx<double>>(cplx<double>*, int64_t, uint64_t, cudaStream_t);
template void launch_philox<cplx<float>>(cplx<float>*, int64_t, uint64_t, cudaStream_t);
template int build_adjoint<double>(int, const int*, const int*, const double*, int**, int**, double**, int*,
                                   int*, cudaStream_t);
template int build_adjoint<float>(int, const int*, const int*, const float*, int**, int**, float**, int*, int*,
                                  cudaStream_t);
template int build_adjoint<cplx<double>>(int, const int*, const int*, const cplx<double>*, int**, int**,
                                         cplx<double>**, int*, int*, cudaStream_t);
template int build_adjoint<cplx<float>>(int, const int*, const int*, const cplx<float>*, int**, int**,
                                        cplx<float>**, int*, int*, cudaStream_t);

}  // namespace rb
