// Smoothed-aggregation multigrid preconditioner for the damped normal
// equations (H + lambda I) delta = rhs of the essential graph (Sec. IV-F's
// linear solve).  Block-Jacobi PCG needs O(N) iterations on the long chains
// of keyframes that loop closing optimises; this hierarchy brings that to a
// few tens, independent of the graph size.
//
// Hierarchy.  Level 0 is the vertex graph.  Aggregates are runs of AMG_M
// consecutive free vertices (keyframe order follows the trajectory, so a
// run is a contiguous piece of it); each aggregate becomes one node of the
// next level with 7 unknowns: the rigid Sim(3) motion of the whole piece.
// Right-multiplying every pose of an aggregate by one G = exp(eps) leaves all
// residuals between them unchanged, and in left-tangent coordinates that
// motion is delta_v = Adj(S_v S_ref^-1) eps' with eps' = Adj(S_ref) eps for a
// reference vertex of the aggregate.  So the tentative prolongation block of
// vertex v is T_v = Adj(S_v S_ref^-1) (the near-null space of the operator);
// coarser levels use the same rule with the reference vertices of the nodes.
// The prolongation is smoothed once, P = (I - 4/(3 rho) D^-1 A) T with rho an
// estimate of the spectral radius of D^-1 A (power iteration), and the coarse
// operator is the Galerkin product P^T A P.  The coarsest level (at most
// AMG_CMAX nodes) is inverted densely.  The preconditioner is one symmetric
// V(1,1) cycle with damped block-Jacobi smoothing, weight 1/rho.
//
// The sparsity of every level and the index lists of every product are built
// once on the host (amg_build); the numeric setup (k_amg_setup) runs on the
// device at every linearisation, because H, lambda and the poses change.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "amg.cuh"
#include "gridsync.cuh"
#include "phases.cuh"

namespace pgo {

// ---------------------------------------------------------------------------
// Host: symbolic hierarchy
// ---------------------------------------------------------------------------

struct AmgHost {
  AmgDev h{};                // descriptor with device pointers (host copy)
  AmgDev* d = nullptr;       // the same descriptor in device memory
  char* mem = nullptr;
  size_t bytes = 0;
};

namespace {

// Allocator whose value-less construct() leaves trivial elements
// uninitialised: the recipe arrays (megabytes on large graphs) are filled by
// the analysis threads in parallel, so zeroing them on resize would be a
// serial pass over fresh pages.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) {}
  template <class U>
  void construct(U* p) noexcept {
    ::new ((void*)p) U;
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    ::new ((void*)p) U(std::forward<Args>(args)...);
  }
};
using Recipe = std::vector<int2, NoInitAlloc<int2>>;

struct HostLevel {
  int n = 0, n_next = 0;
  std::vector<int> ref, refc, agg;
  std::vector<int> a_ptr, a_col, a_src;     // levels >= 1
  std::vector<int> p_ptr, p_col, p_row, pt_ptr, pt_row, pt_blk;
  std::vector<int> ap_ptr, ap_col;
  std::vector<int> ap_row, ap_pblk, apt_ptr, apt_row, apt_blk;   // single-graph hierarchies
  std::vector<int> r1_ptr, r2_ptr, r3_ptr;
  Recipe r1, r2, r3;
  std::vector<int> ord1, ord2, ord1t, ord2t, ord3;   // output blocks by recipe length, longest first
};

// Neighbour terms (A reference, node) of row u, the diagonal first.
// Level 0: A reference -(u+1) is the damped diagonal block of u, a reference
// k >= 0 is incidence code k (stored block k >> 1, transposed if k & 1).
// Levels >= 1: the index of the stored block.
struct NbrView {
  int level;
  const std::vector<char>* fixed;              // level 0: gauge vertices
  const int *inc_ptr, *inc_code, *inc_other;   // level 0
  const std::vector<int>* a_ptr;               // levels >= 1
  const std::vector<int>* a_col;
  template <class F>
  void each(int u, F f) const {
    if (level == 0) {
      if ((*fixed)[u]) return;
      f(-(u + 1), u);
      for (int k = inc_ptr[u]; k < inc_ptr[u + 1]; ++k) {
        const int w = inc_other[k];
        if (!(*fixed)[w]) f(inc_code[k], w);
      }
    } else {
      for (int k = (*a_ptr)[u]; k < (*a_ptr)[u + 1]; ++k) f(k, (*a_col)[k]);
    }
  }
};


// Host worker pool of the hierarchy analysis: created on first use, kept for
// the life of the process (spawning threads per call cost as much as the
// work on a 2,000-keyframe graph).  run(n, f) calls f(0) .. f(n - 1) on the
// workers and the calling thread and returns when all are done; concurrent
// callers take turns.  A process forked after the pool exists has no
// workers: run() then executes the calls itself.
class HostPool {
 public:
  static HostPool& get() {
    static HostPool* p = new HostPool();   // never destroyed: workers idle at exit
    return *p;
  }
  int width() const { return nthreads_ + 1; }
  void run(int n, const std::function<void(int)>& f) {
    std::lock_guard<std::mutex> serial(run_mu_);
    if (n <= 1 || nthreads_ == 0 || getpid() != pid_) {
      for (int i = 0; i < n; ++i) f(i);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &f;
      njobs_ = n;
      next_.store(0);
      pending_ = n;
      ++gen_;
    }
    cv_.notify_all();
    drain();
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return pending_ == 0; });
    job_ = nullptr;
  }

 private:
  HostPool() : pid_(getpid()) {
    const unsigned hw = std::thread::hardware_concurrency();
    nthreads_ = (int)std::min<unsigned>(hw > 1 ? hw - 1 : 0, 15);
    for (int t = 0; t < nthreads_; ++t) std::thread([this] { loop(); }).detach();
  }
  void drain() {
    for (;;) {
      const int i = next_.fetch_add(1);
      if (i >= njobs_) return;
      (*job_)(i);
      std::lock_guard<std::mutex> lk(mu_);
      if (--pending_ == 0) done_cv_.notify_all();
    }
  }
  void loop() {
    unsigned seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
      }
      drain();
    }
  }
  const pid_t pid_;
  int nthreads_ = 0;
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* job_ = nullptr;
  int njobs_ = 0, pending_ = 0;
  unsigned gen_ = 0;
  std::atomic<int> next_{0};
};

// Rows [0, n) of a block-sparse product, grouped by column: gen(row, emit)
// emits terms emit(col, x, y); each row gets its distinct columns ascending
// (plus `diag_col(row)` when that is >= 0) and each (row, column) block its
// terms in emission order.  Output: row pointers, columns, per-block term
// pointers and the terms (int2 {x, y}).  Rows are split into contiguous
// chunks over host threads and the chunks concatenated in order, so the
// result does not depend on the thread count.
template <class Gen, class Diag>
void group_rows(int n, int ncols, Gen gen, Diag diag_col, std::vector<int>& row_ptr, std::vector<int>& col,
                std::vector<int>& rec_ptr, Recipe& rec, size_t n_terms = 0) {
  struct Chunk {
    std::vector<int> row_len, col, blk_len;
    Recipe rec;
  };
  HostPool& pool = HostPool::get();
  int T = std::min(pool.width(), 16);
  if (n < 128) T = 1;
  // the chunk buffers of the calling thread are kept between calls: their
  // pages stay mapped, so later products and later graphs do not fault them
  // in again
  static thread_local std::vector<Chunk> cache;
  if ((int)cache.size() < T) cache.resize(T);
  Chunk* ch = cache.data();
  for (int t = 0; t < T; ++t) {
    ch[t].row_len.clear();
    ch[t].col.clear();
    ch[t].blk_len.clear();
    ch[t].rec.clear();
  }
  auto work = [&](int t) {
    const int r0 = (int)((long long)n * t / T), r1 = (int)((long long)n * (t + 1) / T);
    Chunk& c = ch[t];
    // the chunk's share of the terms, reserved once (growth by doubling
    // copies the terms again and touches fresh pages each time)
    if (n_terms) c.rec.reserve((size_t)((double)n_terms * (r1 - r0) / n * 1.05) + 256);
    c.blk_len.reserve((size_t)(r1 - r0) * 8);
    c.col.reserve((size_t)(r1 - r0) * 8);
    std::vector<int> slot(std::max(ncols, 1), -1), cols, cnt, fill, td;
    std::vector<int2> tv;
    for (int u = r0; u < r1; ++u) {
      td.clear();
      tv.clear();
      gen(u, [&](int d, int x, int y) {
        td.push_back(d);
        tv.push_back(make_int2(x, y));
        if (slot[d] < 0) {
          slot[d] = 0;
          cols.push_back(d);
        }
      });
      const int dc = diag_col(u);
      if (dc >= 0 && slot[dc] < 0) {
        slot[dc] = 0;
        cols.push_back(dc);
      }
      std::sort(cols.begin(), cols.end());
      const int m = (int)cols.size();
      for (int k = 0; k < m; ++k) slot[cols[k]] = k;
      cnt.assign(m + 1, 0);
      for (int d : td) cnt[slot[d] + 1]++;
      for (int k = 0; k < m; ++k) cnt[k + 1] += cnt[k];
      const size_t base = c.rec.size();
      c.rec.resize(base + td.size());
      fill.assign(cnt.begin(), cnt.end() - 1);
      for (size_t q = 0; q < td.size(); ++q) c.rec[base + fill[slot[td[q]]]++] = tv[q];
      for (int k = 0; k < m; ++k) {
        c.col.push_back(cols[k]);
        c.blk_len.push_back(cnt[k + 1] - cnt[k]);
        slot[cols[k]] = -1;
      }
      c.row_len.push_back(m);
      cols.clear();
    }
  };
  pool.run(T, work);
  // concatenate in chunk order: offsets from the chunk sizes, then every
  // chunk copies itself into place on its own thread
  std::vector<size_t> blk0(T + 1, 0), rec0(T + 1, 0);
  for (int t = 0; t < T; ++t) {
    blk0[t + 1] = blk0[t] + ch[t].blk_len.size();
    rec0[t + 1] = rec0[t] + ch[t].rec.size();
  }
  row_ptr.assign(n + 1, 0);
  col.resize(blk0[T]);
  rec_ptr.resize(blk0[T] + 1);
  rec_ptr[0] = 0;
  rec.resize(rec0[T]);
  pool.run(T, [&](int t) {
    const Chunk& c = ch[t];
    const int r0 = (int)((long long)n * t / T);
    int nb = (int)blk0[t];
    for (size_t i = 0; i < c.row_len.size(); ++i) {
      nb += c.row_len[i];
      row_ptr[r0 + i + 1] = nb;
    }
    int nr = (int)rec0[t];
    for (size_t k = 0; k < c.blk_len.size(); ++k) {
      nr += c.blk_len[k];
      rec_ptr[blk0[t] + k + 1] = nr;
    }
    std::copy(c.col.begin(), c.col.end(), col.begin() + blk0[t]);
    std::copy(c.rec.begin(), c.rec.end(), rec.begin() + rec0[t]);
  });
}

// Position `pos` of round k over a list walked `stride` entries per round,
// forwards in even rounds and backwards in odd ones: with the list sorted
// longest first, every worker gets a long and a short entry in turn.
__device__ __forceinline__ int snake(int k, int stride, int pos) {
  return k * stride + ((k & 1) ? stride - 1 - pos : pos);
}

// Block indices ordered by recipe length (ptr[b + 1] - ptr[b]), longest
// first, ties in index order: over the whole list (window 0, a counting
// sort), or within each window of `window` consecutive blocks, which keeps
// the blocks of a row near each other (they share the row's operator blocks
// in L1) while the four blocks a warp takes get similar lengths.  The
// windowed form orders windows [w0, w1) of the list only (parts of one list
// run on several threads); the caller sizes `ord` first.
void order_by_length(const std::vector<int>& ptr, std::vector<int>& ord, int window, int w0 = 0,
                     int w1 = 0x7fffffff) {
  const int nb = (int)ptr.size() - 1;
  if (nb <= 0) return;
  auto len = [&](int b) { return ptr[b + 1] - ptr[b]; };
  if (window > 0) {
    for (int b0 = w0 * window; b0 < nb && b0 / window < w1; b0 += window) {
      const int b1 = std::min(nb, b0 + window);
      int key[64];   // window <= 64
      for (int b = b0; b < b1; ++b) {   // stable insertion sort of the window
        const int lb = len(b);
        int k = b;
        while (k > b0 && key[k - 1 - b0] < lb) {
          ord[k] = ord[k - 1];
          key[k - b0] = key[k - 1 - b0];
          --k;
        }
        ord[k] = b;
        key[k - b0] = lb;
      }
    }
    return;
  }
  int mx = 0;
  for (int b = 0; b < nb; ++b) mx = std::max(mx, len(b));
  std::vector<int> pos(mx + 2, 0);
  for (int b = 0; b < nb; ++b) pos[mx - len(b) + 1]++;
  for (int k = 0; k <= mx; ++k) pos[k + 1] += pos[k];
  for (int b = 0; b < nb; ++b) ord[pos[mx - len(b)]++] = b;
}

// Builds P, AP, the recipes and the pattern of the next level for `L`.
// Recipe entries of an output block keep a fixed order: neighbours in
// incidence order, then the blocks of their rows in column order.
void build_level(HostLevel& L, const NbrView& nb, HostLevel& next, bool dense) {
  const int n = L.n, nn = L.n_next;
  // ---- P pattern (the aggregates of the node and of its neighbours) and R1 ----
  size_t n_nb = 0;   // neighbour terms over all rows (an upper bound of R1)
  for (int u = 0; u < n; ++u) nb.each(u, [&](int, int) { ++n_nb; });
  group_rows(
      n, nn,
      [&](int u, auto emit) {
        if (L.agg[u] < 0) return;
        nb.each(u, [&](int a, int w) {
          if (L.agg[w] >= 0) emit(L.agg[w], a, w);
        });
      },
      [&](int u) { return L.agg[u]; }, L.p_ptr, L.p_col, L.r1_ptr, L.r1, n_nb);
  const int nnz_p = L.p_ptr[n];
  L.p_row.resize(nnz_p);
  for (int u = 0; u < n; ++u)
    for (int k = L.p_ptr[u]; k < L.p_ptr[u + 1]; ++k) L.p_row[k] = u;
  // CSC of P (rows ascending within each column)
  L.pt_ptr.assign(nn + 1, 0);
  for (int k = 0; k < nnz_p; ++k) L.pt_ptr[L.p_col[k] + 1]++;
  for (int c = 0; c < nn; ++c) L.pt_ptr[c + 1] += L.pt_ptr[c];
  L.pt_row.resize(nnz_p);
  L.pt_blk.resize(nnz_p);
  {
    std::vector<int> f(L.pt_ptr.begin(), L.pt_ptr.end() - 1);
    for (int u = 0; u < n; ++u)
      for (int k = L.p_ptr[u]; k < L.p_ptr[u + 1]; ++k) {
        const int x = f[L.p_col[k]]++;
        L.pt_row[x] = u;
        L.pt_blk[x] = k;
      }
  }
  // ---- AP pattern and R2: AP_ud = sum_w A_uw P_wd ----
  size_t n_r2 = 0;   // terms of R2: |P row w| per neighbour w of every row
  for (int u = 0; u < n; ++u)
    if (L.agg[u] >= 0) nb.each(u, [&](int, int w) { n_r2 += (size_t)(L.p_ptr[w + 1] - L.p_ptr[w]); });
  group_rows(
      n, nn,
      [&](int u, auto emit) {
        if (L.agg[u] < 0) return;
        nb.each(u, [&](int a, int w) {
          for (int k = L.p_ptr[w]; k < L.p_ptr[w + 1]; ++k) emit(L.p_col[k], a, k);
        });
      },
      [](int) { return -1; }, L.ap_ptr, L.ap_col, L.r2_ptr, L.r2, n_r2);
  if (dense) {
    // Q = (I - D^-1 A / rho) P lives in the pattern of A P, which contains
    // that of P (A has every diagonal block): the row of each block, the P
    // block at the same place (both rows have ascending columns), the CSC
    const int nnz_ap = L.ap_ptr[n];
    L.ap_row.resize(nnz_ap);
    L.ap_pblk.assign(nnz_ap, -1);
    for (int u = 0; u < n; ++u) {
      int kp = L.p_ptr[u];
      for (int k = L.ap_ptr[u]; k < L.ap_ptr[u + 1]; ++k) {
        L.ap_row[k] = u;
        while (kp < L.p_ptr[u + 1] && L.p_col[kp] < L.ap_col[k]) ++kp;
        if (kp < L.p_ptr[u + 1] && L.p_col[kp] == L.ap_col[k]) L.ap_pblk[k] = kp;
      }
    }
    L.apt_ptr.assign(nn + 1, 0);
    for (int k = 0; k < nnz_ap; ++k) L.apt_ptr[L.ap_col[k] + 1]++;
    for (int c = 0; c < nn; ++c) L.apt_ptr[c + 1] += L.apt_ptr[c];
    L.apt_row.resize(nnz_ap);
    L.apt_blk.resize(nnz_ap);
    std::vector<int> f(L.apt_ptr.begin(), L.apt_ptr.end() - 1);
    for (int u = 0; u < n; ++u)
      for (int k = L.ap_ptr[u]; k < L.ap_ptr[u + 1]; ++k) {
        const int x = f[L.ap_col[k]]++;
        L.apt_row[x] = u;
        L.apt_blk[x] = k;
      }
  }
  // ---- next level: upper half of P^T A P from the products, R3 per upper block ----
  std::vector<int> up_ptr, up_col, up_r3ptr;
  Recipe up_r3;
  size_t n_r3 = 0;   // an upper bound of R3: the whole A P row per P^T entry
  for (int t = 0; t < L.pt_ptr[nn]; ++t) n_r3 += (size_t)(L.ap_ptr[L.pt_row[t] + 1] - L.ap_ptr[L.pt_row[t]]);
  group_rows(
      nn, nn,
      [&](int c, auto emit) {
        for (int t = L.pt_ptr[c]; t < L.pt_ptr[c + 1]; ++t) {
          const int u = L.pt_row[t], pb = L.pt_blk[t];
          for (int k = L.ap_ptr[u]; k < L.ap_ptr[u + 1]; ++k)
            if (L.ap_col[k] >= c) emit(L.ap_col[k], pb, k);
        }
      },
      [](int c) { return c; }, up_ptr, up_col, up_r3ptr, up_r3, n_r3 / 2 + n_r3 / 8);
  // lower half by transposition (rows ascending, so each row's lower columns are ascending)
  std::vector<int> lo_ptr(nn + 1, 0);
  for (int c = 0; c < nn; ++c)
    for (int k = up_ptr[c] + 1; k < up_ptr[c + 1]; ++k) lo_ptr[up_col[k] + 1]++;
  for (int c = 0; c < nn; ++c) lo_ptr[c + 1] += lo_ptr[c];
  std::vector<int> lo_col(lo_ptr[nn]), lo_src(lo_ptr[nn]);   // lower block (d, c): source upper block of row c
  {
    std::vector<int> f(lo_ptr.begin(), lo_ptr.end() - 1);
    for (int c = 0; c < nn; ++c)
      for (int k = up_ptr[c] + 1; k < up_ptr[c + 1]; ++k) {
        const int x = f[up_col[k]]++;
        lo_col[x] = c;
        lo_src[x] = k;   // upper-list index, turned into a block index below
      }
  }
  // row c: the diagonal, the lower columns, then the upper columns (all ascending)
  next.a_ptr.assign(nn + 1, 0);
  for (int c = 0; c < nn; ++c) next.a_ptr[c + 1] = next.a_ptr[c] + (up_ptr[c + 1] - up_ptr[c]) + (lo_ptr[c + 1] - lo_ptr[c]);
  const int nnz_next = next.a_ptr[nn];
  next.a_col.resize(nnz_next);
  next.a_src.assign(nnz_next, -1);
  std::vector<int> up_blk(up_col.size());   // upper-list index -> block index
  for (int c = 0; c < nn; ++c) {
    int b = next.a_ptr[c];
    up_blk[up_ptr[c]] = b;
    next.a_col[b++] = c;
    b += lo_ptr[c + 1] - lo_ptr[c];
    for (int k = up_ptr[c] + 1; k < up_ptr[c + 1]; ++k) {
      up_blk[k] = b;
      next.a_col[b++] = up_col[k];
    }
  }
  for (int c = 0; c < nn; ++c) {
    int b = next.a_ptr[c] + 1;
    for (int x = lo_ptr[c]; x < lo_ptr[c + 1]; ++x, ++b) {
      next.a_col[b] = lo_col[x];
      next.a_src[b] = up_blk[lo_src[x]];
    }
  }
  // R3 per block of the next level: upper blocks carry their entries, lower
  // blocks none.  Row c lists the diagonal, its lower blocks, then its upper
  // columns, and the upper blocks keep their order, so the terms are those of
  // the upper half in the same sequence: only the pointers change.
  L.r3_ptr.assign(nnz_next + 1, 0);
  for (int c = 0; c < nn; ++c) {
    int k = up_ptr[c];
    for (int b = next.a_ptr[c]; b < next.a_ptr[c + 1]; ++b) {
      if (next.a_src[b] < 0) ++k;
      L.r3_ptr[b + 1] = up_r3ptr[k];
    }
  }
  L.r3 = std::move(up_r3);
  // (measured per phase on 2,000- and 8,000-keyframe graphs: the
  // eight-lane products of the P and A P phases gain most from windows of
  // 32, the 64-thread teams and the P^T A P phase, whose mirrored blocks have
  // no terms, from a full sort)
  // (the windowed sorts in parts of their windows, one job each)
  constexpr int kWin = 32, kParts = 6;
  for (std::vector<int>* o : {&L.ord1, &L.ord1t}) o->assign(std::max((int)L.r1_ptr.size() - 1, 0), 0);
  for (std::vector<int>* o : {&L.ord2, &L.ord2t}) o->assign(std::max((int)L.r2_ptr.size() - 1, 0), 0);
  L.ord3.assign(std::max((int)L.r3_ptr.size() - 1, 0), 0);
  const int nw1 = ((int)L.r1_ptr.size() - 1 + kWin - 1) / kWin, nw2 = ((int)L.r2_ptr.size() - 1 + kWin - 1) / kWin;
  HostPool::get().run(3 + 2 * kParts, [&](int k) {
    if (k == 0) order_by_length(L.r1_ptr, L.ord1t, 0);
    else if (k == 1) order_by_length(L.r2_ptr, L.ord2t, 0);
    else if (k == 2) order_by_length(L.r3_ptr, L.ord3, 0);
    else if (k < 3 + kParts) {
      const int p = k - 3;
      order_by_length(L.r1_ptr, L.ord1, kWin, (int)((long long)nw1 * p / kParts), (int)((long long)nw1 * (p + 1) / kParts));
    } else {
      const int p = k - 3 - kParts;
      order_by_length(L.r2_ptr, L.ord2, kWin, (int)((long long)nw2 * p / kParts), (int)((long long)nw2 * (p + 1) / kParts));
    }
  });
}

// Device arrays of the hierarchy in two regions of one allocation: the
// arrays uploaded from the host first (put: index lists, recipes), then the
// ones the device fills (take: blocks, vectors), so that the uploads are one
// contiguous range.
struct Uploader {
  char* base = nullptr;
  size_t put_region = 0;   // bytes of the put region (from a measuring pass)
  size_t put_used = 0, take_used = 0;
  std::vector<std::pair<size_t, std::pair<const void*, size_t>>> copies;   // (offset, (host, bytes))
  static size_t padded(size_t bytes) { return (bytes + 255) & ~size_t(255); }
  size_t used() const { return std::max(put_region, put_used) + take_used; }   // (a measuring pass has no region yet)
  template <class T>
  T* take(size_t count) {
    const size_t bytes = padded(count * sizeof(T));
    T* p = reinterpret_cast<T*>(base ? base + put_region + take_used : nullptr);
    take_used += bytes;
    return p;
  }
  template <class T, class A>
  const T* put(const std::vector<T, A>& v) {
    const size_t count = v.size() > 0 ? v.size() : 1;
    T* p = reinterpret_cast<T*>(base ? base + put_used : nullptr);
    if (base && !v.empty()) copies.push_back({put_used, {v.data(), v.size() * sizeof(T)}});
    put_used += padded(count * sizeof(T));
    return p;
  }
};

// Pinned host staging of the hierarchy upload, kept for the life of the
// process and grown on demand: the put region is packed into it by the
// analysis worker pool and sent in one copy (one pageable copy per array cost
// a few microseconds each, over a hundred arrays per graph).
struct PinnedStage {
  std::mutex mu;
  char* p = nullptr;
  size_t n = 0;
  static PinnedStage& get() {
    static PinnedStage* s = new PinnedStage();   // never freed: reused by later graphs
    return *s;
  }
  bool reserve(size_t bytes) {
    if (bytes <= n) return true;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    if (cudaHostAlloc(reinterpret_cast<void**>(&p), bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    n = bytes;
    return true;
  }
};

// Lays out (base == nullptr: only measures) every device array of the
// hierarchy and records the host-to-device copies.
void layout(Uploader& U, std::vector<HostLevel>& H, int L, int N, const std::vector<int>& seg_off, int nseg,
            AmgDev& D) {
  D.L = L;
  D.nL = H[L].n;
  D.nseg = nseg;
  D.seg_off = U.put(seg_off);
  for (int l = 0; l <= L; ++l) {
    HostLevel& h = H[l];
    AmgLevel& a = D.lv[l];
    std::memset(&a, 0, sizeof(a));
    a.n = h.n;
    a.n_next = h.n_next;
    const size_t n = (size_t)std::max(h.n, 1);
    if (l >= 1) {
      a.nnz_a = h.a_ptr.empty() ? 0 : h.a_ptr[h.n];
      a.a_ptr = U.put(h.a_ptr);
      a.a_col = U.put(h.a_col);
      a.a_src = U.put(h.a_src);
      a.a64 = U.take<double>((size_t)std::max(a.nnz_a, 1) * BLK64);
      a.a32 = U.take<float>((size_t)std::max(a.nnz_a, 1) * BLK32);
      a.dinv64 = U.take<double>(n * BLK64);
      a.dinv32 = U.take<float>(n * BLK32);
      a.vr64 = U.take<double>(n * VEC);
      a.vy64 = U.take<double>(n * VEC);
      a.vr32 = U.take<float>(n * VEC);
      a.vy32 = U.take<float>(n * VEC);
    }
    a.vx64 = U.take<double>(n * VEC);
    a.vx32 = U.take<float>(n * VEC);
    if (l < L) {
      a.pv64 = U.take<double>(n * VEC);
      a.pv32 = U.take<float>(n * VEC);
    }
    if (l >= 1 && l < L) {
      a.vs64 = U.take<double>(n * VEC);
      a.vs32 = U.take<float>(n * VEC);
    }
    if (l < L) {
      a.nnz_p = h.p_ptr[h.n];
      a.nnz_ap = h.ap_ptr[h.n];
      a.nnz_next = H[l + 1].a_ptr[h.n_next];
      a.ref = U.put(h.ref);
      a.refc = U.put(h.refc);
      a.agg = U.put(h.agg);
      a.t64 = U.take<double>(n * BLK64);
      a.t32 = U.take<float>(n * BLK32);
      a.p_ptr = U.put(h.p_ptr);
      a.p_col = U.put(h.p_col);
      a.p_row = U.put(h.p_row);
      a.p64 = U.take<double>((size_t)std::max(a.nnz_p, 1) * BLK64);
      a.p32 = U.take<float>((size_t)std::max(a.nnz_p, 1) * BLK32);
      a.pt_ptr = U.put(h.pt_ptr);
      a.pt_row = U.put(h.pt_row);
      a.pt_blk = U.put(h.pt_blk);
      a.ap_ptr = U.put(h.ap_ptr);
      a.ap_col = U.put(h.ap_col);
      a.ap64 = U.take<double>((size_t)std::max(a.nnz_ap, 1) * BLK64);
      a.ap32 = U.take<float>((size_t)std::max(a.nnz_ap, 1) * BLK32);
      if (nseg == 1) {
        a.ap_row = U.put(h.ap_row);
        a.ap_pblk = U.put(h.ap_pblk);
        a.apt_ptr = U.put(h.apt_ptr);
        a.apt_row = U.put(h.apt_row);
        a.apt_blk = U.put(h.apt_blk);
        a.q64 = U.take<double>((size_t)std::max(a.nnz_ap, 1) * BLK64);
        a.q32 = U.take<float>((size_t)std::max(a.nnz_ap, 1) * BLK32);
      }
      a.r1_ptr = U.put(h.r1_ptr);
      a.r1 = U.put(h.r1);
      a.r2_ptr = U.put(h.r2_ptr);
      a.r2 = U.put(h.r2);
      a.r3_ptr = U.put(h.r3_ptr);
      a.r3 = U.put(h.r3);
      a.ord1 = U.put(h.ord1);
      a.ord2 = U.put(h.ord2);
      a.ord1t = U.put(h.ord1t);
      a.ord2t = U.put(h.ord2t);
      a.ord3 = U.put(h.ord3);
    }
  }
  // one dense coarsest inverse per segment (segment s at s * AMG_CMAX^2 blocks)
  const size_t nl2 = nseg == 1 ? (size_t)D.nL * D.nL : (size_t)nseg * AMG_CMAX * AMG_CMAX;
  D.cinv64 = U.take<double>(std::max(nl2, (size_t)1) * BLK64);
  D.cinv32 = U.take<float>(std::max(nl2, (size_t)1) * BLK32);
  D.dense = nseg == 1 ? 1 : 0;
  if (D.dense) {
    const size_t nd = (size_t)H[L - 1].n;
    D.w64 = U.take<double>(nd * nd * BLK64);
    D.w32 = U.take<float>(nd * nd * BLK32);
    D.h64 = U.take<double>(nd * D.nL * BLK64);
    D.h32 = U.take<float>(nd * D.nL * BLK32);
  }
  D.rho = U.take<double>((size_t)nseg * (AMG_MAXL + 1));
  D.rho_next = U.take<double>((size_t)nseg * (AMG_MAXL + 1));
  for (int k = 0; k < 2; ++k) {
    D.pw64[k] = U.take<double>((size_t)N * VEC);
    D.pw32[k] = U.take<float>((size_t)N * VEC);
  }
  D.flag = U.take<int>(nseg);
  D.warm = U.take<int>(2 * (size_t)nseg);
}

}  // namespace

// Host analysis of a hierarchy (no CUDA call): the levels' patterns and
// recipes, ready for amg_upload.
struct AmgPlan {
  std::vector<HostLevel> H;
  int L = 0, N = 0, nseg = 0;
  std::vector<int> seg_off;
};

void amg_plan_free(AmgPlan* P) { delete P; }

// One integer array of level `level` of an analysed plan, for the host tests:
// 0 the node count of every level (level ignored), 1 aggregates, 2 / 3 the
// CSR of P's pattern, 4 / 5 the CSR of A P's pattern, 6 / 7 the CSR of the
// level's operator pattern (levels >= 1).  Returns the length and points
// *data at the values (valid while the plan lives; the node counts until the
// next call on this thread), or -1 for a level or array that does not exist.
long long amg_plan_array(const AmgPlan* P, int level, int what, const int** data) {
  static thread_local std::vector<int> counts;
  if (what == 0) {
    counts.clear();
    for (const HostLevel& h : P->H) counts.push_back(h.n);
    *data = counts.data();
    return (long long)counts.size();
  }
  if (level < 0 || level >= (int)P->H.size()) return -1;
  const HostLevel& h = P->H[level];
  const std::vector<int>* v = nullptr;
  switch (what) {
    case 1: v = &h.agg; break;
    case 2: v = &h.p_ptr; break;
    case 3: v = &h.p_col; break;
    case 4: v = &h.ap_ptr; break;
    case 5: v = &h.ap_col; break;
    case 6: v = &h.a_ptr; break;
    case 7: v = &h.a_col; break;
    default: return -1;
  }
  *data = v->data();
  return (long long)v->size();
}

AmgPlan* amg_analyze(int N, int nseg, const int* seg_v0, const int* seg_nv, const int* seg_fixed, const int* inc_ptr,
                     const int* inc_code, const int* inc_other, const char** err) {
  *err = nullptr;
  // Segments are independent graphs on consecutive vertex ranges (one for a
  // single graph; one per graph of a batch): aggregates never cross a
  // segment, so every level is block-diagonal over the segments.  All
  // segments coarsen the same number of times, until none has more than
  // AMG_CMAX nodes (a small segment shrinks to one node and stays there).
  std::vector<char> fixed(N, 0);
  int K = 0;
  for (int g = 0; g < nseg; ++g) {
    fixed[seg_fixed[g]] = 1;
    K += seg_nv[g] - 1;
  }
  if (K < 1) {
    *err = "multigrid needs at least one free vertex";
    return nullptr;
  }
  std::vector<HostLevel> H(1);
  std::vector<int> seg_off;                  // (levels) x (nseg + 1) node offsets
  std::vector<int> cnt(nseg), cnt_next(nseg);
  {
    HostLevel& L0 = H[0];
    L0.n = N;
    L0.agg.assign(N, -1);
    L0.ref.resize(N);
    int base = 0;
    for (int g = 0; g < nseg; ++g) {
      int fo = 0;
      for (int v = seg_v0[g]; v < seg_v0[g] + seg_nv[g]; ++v) {
        L0.ref[v] = v;
        if (fixed[v]) continue;
        L0.agg[v] = base + fo / AMG_M;
        ++fo;
      }
      cnt_next[g] = (fo + AMG_M - 1) / AMG_M;
      base += cnt_next[g];
    }
    L0.n_next = base;
    for (int g = 0; g <= nseg; ++g) seg_off.push_back(g < nseg ? seg_v0[g] : N);
  }
  int L = 0;
  for (;;) {
    if (L + 1 > AMG_MAXL) {
      *err = "graph too large for the multigrid hierarchy";
      return nullptr;
    }
    H.emplace_back();
    HostLevel& cur = H[L];       // (emplace_back may move the vector)
    HostLevel& nxt = H[L + 1];
    NbrView nb{L, &fixed, inc_ptr, inc_code, inc_other, &cur.a_ptr, &cur.a_col};
    build_level(cur, nb, nxt, nseg == 1);
    nxt.n = cur.n_next;
    // references: the first member of each aggregate
    nxt.ref.assign(nxt.n, -1);
    for (int u = 0; u < cur.n; ++u) {
      const int c = cur.agg[u];
      if (c >= 0 && nxt.ref[c] < 0) nxt.ref[c] = cur.ref[u];
    }
    cur.refc.assign(cur.n, 0);
    for (int u = 0; u < cur.n; ++u) cur.refc[u] = cur.agg[u] >= 0 ? nxt.ref[cur.agg[u]] : 0;
    ++L;
    cnt = cnt_next;
    {
      int o = 0;
      for (int g = 0; g < nseg; ++g) {
        seg_off.push_back(o);
        o += cnt[g];
      }
      seg_off.push_back(o);
    }
    int most = 0;
    for (int g = 0; g < nseg; ++g) most = std::max(most, cnt[g]);
    if (most <= AMG_CMAX) break;
    nxt.agg.resize(nxt.n);
    int base = 0, o = 0;
    for (int g = 0; g < nseg; ++g) {
      for (int c = 0; c < cnt[g]; ++c) nxt.agg[o + c] = base + c / AMG_M;
      o += cnt[g];
      cnt_next[g] = (cnt[g] + AMG_M - 1) / AMG_M;
      base += cnt_next[g];
    }
    nxt.n_next = base;
  }
  AmgPlan* P = new AmgPlan();
  P->H = std::move(H);
  P->L = L;
  P->N = N;
  P->nseg = nseg;
  P->seg_off = std::move(seg_off);
  return P;
}

// Device allocation and upload of an analysed hierarchy (the plan's host
// arrays must live until this returns; it synchronises the stream).
AmgHost* amg_upload(AmgPlan* P, cudaStream_t s, const char** err) {
  *err = nullptr;
  std::vector<HostLevel>& H = P->H;
  const int L = P->L, N = P->N, nseg = P->nseg;
  const std::vector<int>& seg_off = P->seg_off;
  AmgHost* A = new AmgHost();
  Uploader meas;
  layout(meas, H, L, N, seg_off, nseg, A->h);
  A->bytes = meas.used() + 256;
  if (cudaMalloc(&A->mem, A->bytes) != cudaSuccess ||
      cudaMalloc(&A->d, sizeof(AmgDev)) != cudaSuccess) {
    cudaGetLastError();
    *err = "device allocation for the multigrid hierarchy failed";
    amg_free(A);
    return nullptr;
  }
  Uploader up;
  up.base = A->mem;
  up.put_region = meas.put_used;
  layout(up, H, L, N, seg_off, nseg, A->h);
  const size_t nput = up.put_used;
  bool ok = cudaMemsetAsync(A->mem, 0, up.used(), s) == cudaSuccess;
  PinnedStage& stage = PinnedStage::get();
  std::unique_lock<std::mutex> lk(stage.mu);
  if (ok && nput > 0 && stage.reserve(nput)) {
    // pack the put region (arrays at their offsets, the gaps zero as the
    // memset leaves them), in slices of at most 256 KB over the worker pool
    std::vector<std::pair<size_t, size_t>> gaps;   // (offset, bytes) not covered by a copy
    std::vector<std::pair<size_t, std::pair<const char*, size_t>>> slices;
    size_t at = 0;
    for (auto& c : up.copies) {
      if (c.first > at) gaps.push_back({at, c.first - at});
      const char* src = static_cast<const char*>(c.second.first);
      for (size_t o = 0; o < c.second.second; o += (size_t)256 << 10)
        slices.push_back({c.first + o, {src + o, std::min(c.second.second - o, (size_t)256 << 10)}});
      at = c.first + c.second.second;
    }
    if (nput > at) gaps.push_back({at, nput - at});
    for (auto& gp : gaps) std::memset(stage.p + gp.first, 0, gp.second);
    HostPool::get().run((int)slices.size(), [&](int k) {
      std::memcpy(stage.p + slices[k].first, slices[k].second.first, slices[k].second.second);
    });
    ok = cudaMemcpyAsync(A->mem, stage.p, nput, cudaMemcpyHostToDevice, s) == cudaSuccess;
  } else {
    for (auto& c : up.copies)
      ok = ok && cudaMemcpyAsync(A->mem + c.first, c.second.first, c.second.second, cudaMemcpyHostToDevice, s) ==
                     cudaSuccess;
  }
  ok = ok && cudaMemcpyAsync(A->d, &A->h, sizeof(AmgDev), cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(s) == cudaSuccess;   // the host vectors (and the stage) are free again
  lk.unlock();
  if (!ok) {
    *err = "uploading the multigrid hierarchy failed";
    amg_free(A);
    return nullptr;
  }
  return A;
}

AmgHost* amg_build(int N, int nseg, const int* seg_v0, const int* seg_nv, const int* seg_fixed, const int* inc_ptr,
                   const int* inc_code, const int* inc_other, cudaStream_t s, const char** err) {
  AmgPlan* P = amg_analyze(N, nseg, seg_v0, seg_nv, seg_fixed, inc_ptr, inc_code, inc_other, err);
  if (!P) return nullptr;
  AmgHost* A = amg_upload(P, s, err);
  amg_plan_free(P);
  return A;
}

void amg_free(AmgHost* h) {
  if (!h) return;
  if (h->mem) cudaFree(h->mem);
  if (h->d) cudaFree(h->d);
  delete h;
}
const AmgDev* amg_host_desc(const AmgHost* h) { return h ? &h->h : nullptr; }
const AmgDev* amg_device_desc(const AmgHost* h) { return h ? h->d : nullptr; }
size_t amg_bytes(const AmgHost* h) { return h ? h->bytes : 0; }

// ---------------------------------------------------------------------------
// Device: numeric setup
// ---------------------------------------------------------------------------

// A block of level l for a recipe reference: entry (i, k) is
// (tr ? p[k * 7 + i] : p[i * 7 + k]) + (i == k ? add : 0).
// Per-block partial (one double per block) and its fixed-order grid sum,
// double-buffered by `set` so that a fast block's next write cannot race a
// slow block's read.
// The square root of the fixed-order grid sum of the per-block partials
// (0 for a zero or non-finite sum) and its reciprocal (0 for 0), formed once
// per block: FP64 square roots and divisions by every thread of the block
// would cost microseconds at the FP64 rate.
__device__ __forceinline__ double2 grid_norm_after_sync(const double* partial) {
  __shared__ double2 res;
  if (threadIdx.x < 32) {
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int b = threadIdx.x + 32 * q;
      v[q] = b < (int)gridDim.x ? __ldcg(partial + b) : 0.0;
    }
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += v[q];
    for (int b = threadIdx.x + 256; b < (int)gridDim.x; b += 32) acc += __ldcg(partial + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) {
      double nx = sqrt(acc);
      if (!(nx > 0.0) || !isfinite(nx)) nx = 0.0;
      res = make_double2(nx, nx > 0.0 ? 1.0 / nx : 0.0);
    }
  }
  __syncthreads();
  const double2 r = res;
  __syncthreads();
  return r;
}

__device__ __forceinline__ void block_partial(double v, double* partial) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
  __syncthreads();
}

// Barrier of the 64 threads (two warps) of team `slot` (named barriers 1..8
// for the at most 8 teams of a block; barrier 0 is __syncthreads).
__device__ __forceinline__ void team_sync(int slot) {
  asm volatile("bar.sync %0, 64;" ::"r"(slot + 1) : "memory");
}

// y = D^-1 A (sc x) for the rows of level l, one warp per row: the lanes
// take whole blocks of the row (the diagonal block first, each block in
// 16-byte vector loads), the warp sums
// the partial products, lanes 0..6 apply D^-1.  Returns the thread's part of
// |y|^2.
template <class V>
__device__ double power_step(const DevGraph& g, const AmgLevel& Lv, int l, V lam, const V* x, V sc, V* y) {
  constexpr int BLK = AV<V>::BLK;
  const int n = Lv.n;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  double nrm = 0.0;
  for (int u0 = 0; u0 < n; u0 += warps) {
    const int u = u0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u >= n) continue;   // whole warps leave together
    const bool live = !(l == 0 && u == g.fixed);
    V acc[7];
#pragma unroll
    for (int a = 0; a < 7; ++a) acc[a] = V(0);
    if (live) {
      if (l == 0) {
        const int k0 = __ldg(g.inc_ptr + u), ks = __ldg(g.inc_split + u), k1 = __ldg(g.inc_ptr + u + 1);
        for (int k = k0 - 1 + lane; k < k1; k += 32) {
          int w = u, code = 0;
          const V* B;
          if (k < k0) {
            B = AV<V>::diag(g) + (size_t)u * BLK;
          } else {
            code = __ldg(g.inc_code + k);
            w = __ldg(g.inc_other + k);
            B = AV<V>::off(g) + (size_t)(code >> 1) * BLK;
          }
          V xv[7], Bv[49];
#pragma unroll
          for (int c = 0; c < 7; ++c) xv[c] = sc * __ldcg(x + (size_t)w * VEC + c);
          ld_block<true>(B, Bv);
          const bool tr = k >= ks;
#pragma unroll
          for (int a = 0; a < 7; ++a) {
            V t = (k < k0) ? lam * xv[a] : V(0);
#pragma unroll
            for (int c = 0; c < 7; ++c) t += (tr ? Bv[c * 7 + a] : Bv[a * 7 + c]) * xv[c];
            acc[a] += t;
          }
        }
      } else {
        const V* Ab = AV<V>::a(Lv);
        const int k1 = __ldg(Lv.a_ptr + u + 1);
        for (int k = __ldg(Lv.a_ptr + u) + lane; k < k1; k += 32) {
          const int w = __ldg(Lv.a_col + k);
          V xv[7], Bv[49];
#pragma unroll
          for (int c = 0; c < 7; ++c) xv[c] = sc * __ldcg(x + (size_t)w * VEC + c);
          ld_block<false>(Ab + (size_t)k * BLK, Bv);
#pragma unroll
          for (int a = 0; a < 7; ++a) {
            V t = V(0);
#pragma unroll
            for (int c = 0; c < 7; ++c) t += Bv[a * 7 + c] * xv[c];
            acc[a] += t;
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 7; ++a)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    // y = D^-1 acc (lane a < 7 owns component a; lane 7 writes the pad)
    if (lane < 8) {
      V yv = V(0);
      if (lane < 7 && live) {
        const V* M = l == 0 ? AV<V>::minv(g) + (size_t)u * BLK : AV<V>::dinv(Lv) + (size_t)u * BLK;
#pragma unroll
        for (int c = 0; c < 7; ++c) yv += __ldcg(M + lane * 7 + c) * acc[c];
      }
      y[(size_t)u * VEC + lane] = yv;
      nrm += (double)yv * (double)yv;
    }
  }
  return nrm;
}

// Dense copy of the coarsest operator (n7 x n7, row-major) in shared
// memory, every (block, entry) pair at once.
template <class V, class W>
__device__ __forceinline__ void coarsest_dense(const AmgLevel& Lc, W* dense) {
  constexpr int BLK = AV<V>::BLK;
  const int nL = Lc.n, n7 = 7 * nL;
  const V* Ab = AV<V>::a(Lc);
  for (int t = threadIdx.x; t < n7 * n7; t += blockDim.x) dense[t] = W(0);
  __syncthreads();
  const int nnzL = __ldg(Lc.a_ptr + nL);
  for (int t = threadIdx.x; t < nnzL * 49; t += blockDim.x) {
    const int k = t / 49, ij = t - 49 * k;
    int c = 0;
    while (c + 1 < nL && __ldg(Lc.a_ptr + c + 1) <= k) ++c;
    const int d = __ldg(Lc.a_col + k);
    const int i = ij / 7, j = ij - 7 * (ij / 7);
    dense[(7 * c + i) * n7 + 7 * d + j] = W(__ldcg(Ab + (size_t)k * BLK + ij));
  }
  __syncthreads();
}

// Gauss-Jordan inverse of the SPD n7 x n7 matrix in shared memory (no
// pivoting), double-buffered: step k reads buffer k % 2 and writes the other,
// every thread forms the pivot's reciprocal itself, so a step is one block
// barrier (the matrix's row and column k are read from the previous buffer
// while the new one is written).  Element (i, j) goes to thread
// (i mod rows, j mod 64) of the block seen as rows x 64.  The inverse ends in
// the buffer returned (dense or dense + n7 * n7); nullptr on a non-positive or
// non-finite pivot.
template <class W>
__device__ W* gauss_jordan_spd(W* dense, int n7) {
  const int j0 = threadIdx.x & 63, i0 = threadIdx.x >> 6, istep = blockDim.x >> 6;
  W* in = dense;
  W* out = dense + (size_t)n7 * n7;
  for (int k = 0; k < n7; ++k) {
    const W piv = in[k * n7 + k];
    if (!(piv > W(0) && isfinite(piv))) return nullptr;   // uniform: every thread reads the same value
    const W ip = W(1) / piv;
    for (int i = i0; i < n7; i += istep) {
      const W cik = in[i * n7 + k];
      for (int j = j0; j < n7; j += 64) {
        W o;
        if (i == k) o = (j == k) ? ip : in[k * n7 + j] * ip;
        else o = (j == k) ? -cik * ip : in[i * n7 + j] - cik * (in[k * n7 + j] * ip);
        out[i * n7 + j] = o;
      }
    }
    __syncthreads();
    W* t = in;
    in = out;
    out = t;
  }
  return in;
}

// C^-1 of the coarsest level into AV<V>::cinv (symmetrised; zero and the
// failure flag set when a pivot fails).  FP64 elimination for the FP64 set-up.
__device__ void coarsest_inverse_f64(const AmgDev& A, double* dense) {
  const AmgLevel& Lc = A.lv[A.L];
  const int nL = Lc.n, n7 = 7 * nL;
  coarsest_dense<double, double>(Lc, dense);
  const double* inv = gauss_jordan_spd<double>(dense, n7);
  const bool ok = inv != nullptr;
  if (!ok) inv = dense;
  double* Ci = AV<double>::cinv(A);
  for (int t = threadIdx.x; t < nL * nL * 49; t += blockDim.x) {
    const int cd = t / 49, ij = t - 49 * cd;
    const int c = cd / nL, d = cd - nL * c;
    const int i = ij / 7, j = ij - 7 * (ij / 7);
    const int R = 7 * c + i, C = 7 * d + j;
    Ci[(size_t)cd * BLK64 + ij] = ok ? 0.5 * (inv[R * n7 + C] + inv[C * n7 + R]) : 0.0;
  }
  if (threadIdx.x == 0 && !ok) *A.flag = 1;
}

// The FP32 set-up: the elimination in FP32 on the symmetrically Jacobi-scaled
// matrix S C S (unit diagonal, S = diag(C)^-1/2), C^-1 = S (S C S)^-1 S.  At
// GB300's FP64 rate the FP64 elimination of a 56 x 56 matrix takes about
// 0.2 ms on one SM; the scaling keeps the FP32 elimination's error at the
// scaled matrix's condition number, and the operator itself comes from FP32
// products.
// Inverse of one SPD 7x7 block by Gauss-Jordan on a warp: lane r < 7 holds
// row r of [B | I] in registers, the pivot row goes round by shuffles.
// Returns false on a non-positive or non-finite pivot (every lane).
__device__ __forceinline__ bool inv7_warp(const float* B, float* out) {
  const int lane = threadIdx.x & 31;
  float a[7], e[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    a[c] = lane < 7 ? B[lane * 7 + c] : 0.f;
    e[c] = (lane == c) ? 1.f : 0.f;
  }
  bool ok = true;
#pragma unroll
  for (int p = 0; p < 7; ++p) {
    float pa[7], pe[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      pa[c] = __shfl_sync(0xffffffffu, a[c], p);
      pe[c] = __shfl_sync(0xffffffffu, e[c], p);
    }
    const float piv = pa[p];
    ok = ok && piv > 0.f && isfinite(piv);
    const float ip = piv > 0.f ? 1.f / piv : 0.f;
    const float f = (lane == p) ? 0.f : a[p];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      if (lane == p) {
        a[c] *= ip;
        e[c] *= ip;
      } else {
        a[c] -= f * (pa[c] * ip);
        e[c] -= f * (pe[c] * ip);
      }
    }
  }
  if (lane < 7)
#pragma unroll
    for (int c = 0; c < 7; ++c) out[lane * 7 + c] = e[c];
  return ok;
}

// C^-1 of the coarsest level for the FP32 set-up, on the Jacobi-scaled
// operator S C S (unit diagonal): Gauss-Jordan over 7x7 blocks, nL steps of
// three block barriers each -- the pivot block's inverse on warp 0, the
// scaled pivot row R = P M_k* with the pivot column saved, then every block
// M_ij -= M_ik R_j (the pivot column -M_ik P, the pivot row R).
__device__ void coarsest_inverse_f32(const AmgDev& A, float* dense) {
  const AmgLevel& Lc = A.lv[A.L];
  const int nL = Lc.n, n7 = 7 * nL;
  coarsest_dense<float, float>(Lc, dense);
  float* sc = dense + 2 * (size_t)n7 * n7;
  for (int i = threadIdx.x; i < n7; i += blockDim.x) {
    const float d = dense[i * n7 + i];
    sc[i] = d > 0.f && isfinite(d) ? rsqrtf(d) : 1.f;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n7 * n7; t += blockDim.x) {
    const int i = t / n7, j = t - n7 * i;
    dense[t] *= sc[i] * sc[j];
  }
  __syncthreads();
  float* M = dense;
  float* R = dense + (size_t)n7 * n7;   // 7 x n7: the scaled pivot row
  float* Cc = R + 7 * (size_t)n7;       // n7 x 7: the pivot column before the step
  float* Pv = Cc + 7 * (size_t)n7;      // 7 x 7: the pivot block's inverse
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int kb = 0; kb < nL; ++kb) {
    const int k7 = 7 * kb;
    if (threadIdx.x < 32) {
      // gather the pivot block into Pv first (rows of M are n7 apart)
      if (threadIdx.x < 7)
#pragma unroll
        for (int c = 0; c < 7; ++c) Pv[threadIdx.x * 7 + c] = M[(size_t)(k7 + threadIdx.x) * n7 + k7 + c];
      __syncwarp();
      const bool ok = inv7_warp(Pv, Pv);
      if (threadIdx.x == 0 && !ok) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) break;   // uniform
    for (int t = threadIdx.x; t < 7 * n7; t += blockDim.x) {
      const int a = t / n7, J = t - n7 * a;
      float v;
      if (J >= k7 && J < k7 + 7) {
        v = Pv[a * 7 + (J - k7)];
      } else {
        v = 0.f;
#pragma unroll
        for (int q = 0; q < 7; ++q) v += Pv[a * 7 + q] * M[(size_t)(k7 + q) * n7 + J];
      }
      R[t] = v;
      const int I = t / 7, q = t - 7 * I;   // the same 7 n7 entries as the pivot column
      Cc[t] = M[(size_t)I * n7 + k7 + q];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n7 * n7; t += blockDim.x) {
      const int I = t / n7, J = t - n7 * I;
      float v;
      if (I >= k7 && I < k7 + 7) {
        v = R[(I - k7) * n7 + J];
      } else if (J >= k7 && J < k7 + 7) {
        v = 0.f;
#pragma unroll
        for (int q = 0; q < 7; ++q) v -= Cc[I * 7 + q] * Pv[q * 7 + (J - k7)];
      } else {
        v = M[t];
#pragma unroll
        for (int q = 0; q < 7; ++q) v -= Cc[I * 7 + q] * R[q * n7 + J];
      }
      M[t] = v;
    }
    __syncthreads();
  }
  const bool ok = !s_bad;
  float* Ci = AV<float>::cinv(A);
  for (int t = threadIdx.x; t < nL * nL * 49; t += blockDim.x) {
    const int cd = t / 49, ij = t - 49 * cd;
    const int c = cd / nL, d = cd - nL * c;
    const int i = ij / 7, j = ij - 7 * (ij / 7);
    const int Rr = 7 * c + i, C = 7 * d + j;
    Ci[(size_t)cd * BLK32 + ij] = ok ? 0.5f * (M[Rr * n7 + C] + M[C * n7 + Rr]) * sc[Rr] * sc[C] : 0.f;
  }
  if (threadIdx.x == 0 && !ok) *A.flag = 1;
}

// The FP32 products run eight lanes per output block where a phase has at
// least kRowLanesMin output blocks; below that the 64-thread teams (one
// output entry per thread) are faster: all their blocks fit in one pass of
// the grid, and a team's term costs 7 FMA where a lane's costs 49.
constexpr int kRowLanesMin = 4096;
template <class V>
__device__ __forceinline__ bool row_lanes(int n_out) {
  return sizeof(V) == 4 && n_out >= kRowLanesMin;
}

// ---- FP32 block products, one lane per output row --------------------------
// Eight lanes take one 7x7 output block (lane r < 7 its row r, lane 7 idle),
// four blocks per warp.  Per recipe term a lane holds the whole right operand
// block in registers (sixteen-byte loads, the same addresses on the block's
// lanes) and streams its row of the left operand, so a term costs 20 loads
// and 49 FMA per lane.
template <bool NC>
__device__ __forceinline__ float4 ld4(const float* p) {
  return NC ? __ldg(reinterpret_cast<const float4*>(p)) : __ldcg(reinterpret_cast<const float4*>(p));
}

template <bool NC>
__device__ __forceinline__ void ld_x52(const float* p, float (&X)[52]) {
#pragma unroll
  for (int ch = 0; ch < 13; ++ch) {
    const float4 v = ld4<NC>(p + 4 * ch);
    X[4 * ch] = v.x;
    X[4 * ch + 1] = v.y;
    X[4 * ch + 2] = v.z;
    X[4 * ch + 3] = v.w;
  }
}

template <bool NC>
__device__ __forceinline__ float ld1(const float* p) {
  return NC ? __ldg(p) : __ldcg(p);
}

// acc[j] += sum_k op(A)[r][k] X[k][j]; op(A) = A, or A^T when TR
template <bool NC, bool TR>
__device__ __forceinline__ void mac_row(const float* A, int r, const float (&X)[52], float (&acc)[7]) {
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const float a = ld1<NC>(A + (TR ? k * 7 + r : r * 7 + k));
#pragma unroll
    for (int j = 0; j < 7; ++j) acc[j] += a * X[k * 7 + j];
  }
}

// row r of the sum over the recipe terms (a, x) of op(A_a) X_x, with A the
// level's operator: at level 0 a < 0 is the damped diagonal block of vertex
// -a - 1 and a >= 0 the stored off-diagonal block a >> 1 (transposed if
// a & 1); at the coarser levels a indexes the level's own (full-row) blocks.
__device__ __forceinline__ void recipe_row_f32(const DevGraph& g, const AmgLevel& Lv, int l, float lam,
                                               const int2* rec, int e0, int e1, const float* X0, int r,
                                               float (&acc)[7]) {
  for (int e = e0; e < e1; ++e) {
    const int2 t = __ldg(rec + e);
    const float* Xp = X0 + (size_t)t.y * BLK32;
    float X[52];
    ld_x52<false>(Xp, X);
    if (l == 0) {
      if (t.x < 0) {
        mac_row<true, false>(g.diag32 + (size_t)(-t.x - 1) * BLK32, r, X, acc);
#pragma unroll
        for (int j = 0; j < 7; ++j) acc[j] += lam * ld1<false>(Xp + r * 7 + j);
      } else if (t.x & 1) {
        mac_row<true, true>(g.off32 + (size_t)(t.x >> 1) * BLK32, r, X, acc);
      } else {
        mac_row<true, false>(g.off32 + (size_t)(t.x >> 1) * BLK32, r, X, acc);
      }
    } else {
      mac_row<false, false>(Lv.a32 + (size_t)t.x * BLK32, r, X, acc);
    }
  }
}

// row r of Y - f M B, with B's rows held by the eight lanes of this block
// (row k in lane base + k) and M a block in memory; Y: a block or nullptr.
template <bool NC>
__device__ __forceinline__ void smooth_row(const float* M, const float* Y, float f, int r, int base,
                                           const float (&b)[7], float (&out)[7]) {
  float s[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) s[j] = 0.f;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const float m = M ? ld1<NC>(M + r * 7 + k) : 0.f;
#pragma unroll
    for (int j = 0; j < 7; ++j) s[j] += m * __shfl_sync(0xffffffffu, b[j], base + k);
  }
#pragma unroll
  for (int j = 0; j < 7; ++j) out[j] = (Y ? ld1<false>(Y + r * 7 + j) : 0.f) - f * s[j];
}

// Block shape of the set-up: 64-thread teams (one 7x7 output block each)
// for the per-node D^-1 inverses and the FP64 products, eight lanes per
// output block for the FP32 products.  FP32 runs 8 teams per block (more
// loads in flight per SM); FP64 runs 4, which leaves it the registers of its
// unrolled products.
template <class V>
struct SetupShape {
  static constexpr int THREADS = sizeof(V) == 4 ? 512 : 256;
  static constexpr int TEAMS = THREADS / 64;
};

// lm: the set-up of an LM iteration.  With DevOptions::amg_refresh = k > 1,
// only every k-th such set-up rebuilds the coarse levels; the others refresh
// the finest level (its smoothing weight, P and A P) and keep the coarse
// levels and the coarsest inverse of the last complete set-up, which stay
// consistent among themselves, so the cycle stays symmetric positive definite.
template <class V>
__global__ void __launch_bounds__(SetupShape<V>::THREADS, 1) k_amg_setup(DevGraph g, int lm) {
  constexpr int TEAMS = SetupShape<V>::TEAMS;
  SolverState* st = g.st;
  if (st->done) return;
  // the hierarchy descriptor, cached in shared memory
  __shared__ AmgDev sA;
  {
    static_assert(sizeof(AmgDev) % 8 == 0, "descriptor copy by 8-byte words");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(g.amg);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sA);
    for (int t = threadIdx.x; t < (int)(sizeof(AmgDev) / 8); t += blockDim.x) dst[t] = src[t];
    __syncthreads();
  }
  const AmgDev& A = sA;
  unsigned* counter = &st->ticket[T_AMG];
  int* abort_flag = reinterpret_cast<int*>(&st->ticket[T_AMG_ABORT]);
  unsigned target = 0;
  constexpr int BLK = AV<V>::BLK;
  const V lam = V(st->lambda);
  const int cur = st->cur;
  const int warm_slot = sizeof(V) == sizeof(double) ? 0 : 1;
  const bool warm = __ldcg(g.amg->warm + warm_slot) != 0;
  const int refresh = g.opt->amg_refresh;
  const bool lagged = lm && warm && refresh > 1 && (st->it % refresh) != 0;
  double* partial = g.partial;
  __shared__ V sacc[TEAMS][49];
  __shared__ double smat[TEAMS][52];   // D^-1 teams (51 doubles each)
  __shared__ double rho_f[2];          // 4 / (3 rho), 1 / rho of the current level
  extern __shared__ double dense[];   // coarsest operator (block 0 only)

  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gthreads = gridDim.x * blockDim.x;
  // ---- tentative prolongation blocks T = Adj(S_ref S_refc^-1), all levels ----
  // one node per thread over the levels' nodes in sequence, node
  // q * gridDim.x + b to block b: each node is a chain of a few hundred
  // dependent FP64 operations, so no thread takes two and every SM takes some.
  // The threads after them form the level-0 smoother blocks
  // D0^-1 = (H_vv + lambda I)^-1, one vertex each (the block-Jacobi
  // preconditioner's kernel is not launched before a multigrid set-up).
  {
    const int nlev = lagged ? 1 : A.L;
    int total = 0;
    for (int l = 0; l < nlev; ++l) total += A.lv[l].n;
    for (int q = threadIdx.x * gridDim.x + blockIdx.x; q < total + g.N; q += gthreads) {
      if (q >= total) {
        const int v = q - total;
        precond_vertex<V>(g, v, g.fixed, st->lambda, const_cast<V*>(AV<V>::minv(g)) + (size_t)v * BLK);
        continue;
      }
      int l = 0, u = q;
      while (u >= A.lv[l].n) {
        u -= A.lv[l].n;
        ++l;
      }
      const AmgLevel& Lv = A.lv[l];
      if (__ldg(Lv.agg + u) < 0) continue;
      const Sim3T<double> Sr = load_pose(g, cur, __ldg(Lv.ref + u));
      const Sim3T<double> Sc = load_pose(g, cur, __ldg(Lv.refc + u));
      double T[7][7];
      adj7(compose(Sr, inverse(Sc)), T);
      V* out = AV<V>::t(Lv) + (size_t)u * BLK;
#pragma unroll
      for (int i = 0; i < 7; ++i)
#pragma unroll
        for (int j = 0; j < 7; ++j) out[i * 7 + j] = V(T[i][j]);
    }
    if (gtid == 0) *A.flag = 0;
  }
  if (!grid_sync(counter, abort_flag, target)) goto timeout;

  for (int l = 0; l < (lagged ? 1 : A.L); ++l) {
    const AmgLevel& Lv = A.lv[l];
    const AmgLevel& Ln = A.lv[l + 1];
    // ---- rho(D^-1 A) ----
    // A warm set-up takes the estimate the previous set-up refined (H, lambda
    // and the poses change little between linearisations; never below the rho
    // of the previous hierarchy) and refines it for the next one with three
    // power steps that ride along with the P, A P and P^T A P phases below, so
    // they add no grid barrier.  The first set-up of a graph (and a lagged
    // one) runs its power iteration in phases of its own.
    double rho;
    const bool fuse = warm && !lagged;
    V* pv = AV<V>::pv(Lv);
    if (fuse) {
      const double rho_prev = __ldcg(A.rho + l), rho_est = __ldcg(A.rho_next + l);
      rho = rho_prev;
      if (rho_est > rho && isfinite(rho_est)) rho = rho_est;
      if (!(rho > 1e-30) || !isfinite(rho)) rho = 1.0;
      // (A.rho[l] is written in the A P phase, after every block has read it)
      if (threadIdx.x == 0) {
        rho_f[0] = 4.0 / (3.0 * rho);
        rho_f[1] = 1.0 / rho;
      }
      __syncthreads();
    } else {
      // start from the vector the previous set-up of this graph ended with,
      // else from a fixed smooth vector
      V* x0 = AV<V>::pw(A, 0);
      const double rho_prev = __ldcg(A.rho + l);   // written after the barriers below
      double nrm = 0.0;
      for (int t = gtid; t < Lv.n * VEC; t += gthreads) {
        const int u = t / VEC, k = t - u * VEC;
        const bool on = k < 7 && !(l == 0 && u == g.fixed);
        double v = 0.0;
        if (on) v = warm ? (double)__ldcg(pv + t) : 1.0 + 0.5 * sin(0.7 * (double)(7 * u + k));
        x0[t] = V(v);
        nrm += v * v;
      }
      block_partial(nrm, partial);
      if (!grid_sync(counter, abort_flag, target)) goto timeout;
      double2 nn = grid_norm_after_sync(partial);   // (|x|, 1 / |x|)
      const int its = warm ? AMG_POWER_ITS_WARM : AMG_POWER_ITS;
      for (int it = 0; it < its; ++it) {
        const V* xin = AV<V>::pw(A, it & 1);
        V* yout = AV<V>::pw(A, (it + 1) & 1);
        double ny2 = power_step<V>(g, Lv, l, lam, xin, V(nn.y), yout);
        double* pset = partial + ((it + 1) & 1) * gridDim.x;
        block_partial(ny2, pset);
        if (!grid_sync(counter, abort_flag, target)) goto timeout;
        nn = grid_norm_after_sync(pset);
      }
      rho = nn.x > 1e-30 ? nn.x : 1.0;
      // a few warm iterations approach rho from below; never go under the
      // previous estimate (an underestimate weakens the smoother's damping)
      if (warm && rho_prev > rho && isfinite(rho_prev)) rho = rho_prev;
      if (gtid == 0) {
        A.rho[l] = rho;
        A.rho_next[l] = rho;
      }
      // the smoother's factors, divided once per block
      if (threadIdx.x == 0) {
        rho_f[0] = 4.0 / (3.0 * rho);
        rho_f[1] = 1.0 / rho;
      }
      __syncthreads();
      const V* yl = AV<V>::pw(A, its & 1);
      for (int t = gtid; t < Lv.n * VEC; t += gthreads) pv[t] = __ldcg(yl + t);
    }
    // ---- P = T_agg - 4/(3 rho) D^-1 (A T) ----
    if (fuse) {   // power step 1: y1 = D^-1 A pv
      const double ny2 = power_step<V>(g, Lv, l, lam, pv, V(1), AV<V>::pw(A, 0));
      block_partial(ny2, partial);
    }
    if (row_lanes<V>(Lv.nnz_p)) {
      if constexpr (sizeof(V) == 4) {
        // FP32: eight lanes per P block, lane r its row
        const float f = (float)rho_f[0];
        const float* Tb = Lv.t32;
        float* Pb = Lv.p32;
        const int lane = threadIdx.x & 31, r = lane & 7, gbase = lane & 24;
        const int stride = (gthreads >> 5) << 2, pos = ((gtid >> 5) << 2) + (lane >> 3);
        for (int k = 0; k * stride < Lv.nnz_p; ++k) {
          const int bi = snake(k, stride, pos);
          const bool on = bi < Lv.nnz_p && r < 7;
          const int b = bi < Lv.nnz_p ? __ldg(Lv.ord1 + bi) : 0;
          float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          int u = 0, c = -1;
          if (on) {
            u = __ldg(Lv.p_row + b);
            c = __ldg(Lv.p_col + b);
            recipe_row_f32(g, Lv, l, (float)lam, Lv.r1, __ldg(Lv.r1_ptr + b), __ldg(Lv.r1_ptr + b + 1), Tb, r, acc);
          }
          const float* M = on ? (l == 0 ? g.minv32 : Lv.dinv32) + (size_t)u * BLK32 : nullptr;
          const float* Y = (on && c == __ldg(Lv.agg + u)) ? Tb + (size_t)u * BLK32 : nullptr;
          float out[7];
          if (l == 0) smooth_row<true>(M, Y, f, r, gbase, acc, out);
          else smooth_row<false>(M, Y, f, r, gbase, acc, out);
          if (on)
#pragma unroll
            for (int jj = 0; jj < 7; ++jj) Pb[(size_t)b * BLK32 + r * 7 + jj] = out[jj];
        }
      }
    } else {
      const double f = rho_f[0];
      const int slot = threadIdx.x >> 6, t = threadIdx.x & 63;
      const int i = t / 7, j = t - 7 * (t / 7);
      const bool lane_on = t < 49;
      const V* Tb = AV<V>::t(Lv);
      V* Pb = AV<V>::p(Lv);
      const int stride = gridDim.x * TEAMS, pos = blockIdx.x * TEAMS + slot;
      for (int k = 0; k * stride < Lv.nnz_p; ++k) {
        const int bi = snake(k, stride, pos);
        const bool has = bi < Lv.nnz_p;
        const int b = has ? __ldg(Lv.ord1t + bi) : 0;
        int u = 0, c = 0;
        if (has && lane_on) {
          u = __ldg(Lv.p_row + b);
          c = __ldg(Lv.p_col + b);
          const int e0 = __ldg(Lv.r1_ptr + b), e1 = __ldg(Lv.r1_ptr + b + 1);
          sacc[slot][t] = l == 0 ? recipe_ax<V, true>(g, nullptr, lam, Lv.r1, e0, e1, Tb, i, j)
                                 : recipe_ax<V, false>(g, AV<V>::a(Lv), lam, Lv.r1, e0, e1, Tb, i, j);
        }
        __syncthreads();
        if (has && lane_on) {
          const V* M = (l == 0 ? AV<V>::minv(g) : AV<V>::dinv(Lv)) + (size_t)u * BLK;
          V s = V(0);
#pragma unroll
          for (int k = 0; k < 7; ++k) s += __ldcg(M + i * 7 + k) * sacc[slot][k * 7 + j];
          const V tv = (c == __ldg(Lv.agg + u)) ? __ldcg(Tb + (size_t)u * BLK + i * 7 + j) : V(0);
          Pb[(size_t)b * BLK + i * 7 + j] = tv - V(f) * s;
        }
        __syncthreads();
      }
    }
    if (!grid_sync(counter, abort_flag, target)) goto timeout;
    // ---- AP = A P; single-graph hierarchies also Q = P - D^-1 (A P) / rho,
    // from the team's AP block in shared memory (a 64-thread barrier per team) ----
    if (fuse) {   // power step 2: y2 = D^-1 A y1 / |y1|; every block has read A.rho[l]
      const double2 nn = grid_norm_after_sync(partial);
      const double ny2 = power_step<V>(g, Lv, l, lam, AV<V>::pw(A, 0), V(nn.y), AV<V>::pw(A, 1));
      block_partial(ny2, partial + gridDim.x);
      if (gtid == 0) A.rho[l] = rho;
    }
    if (row_lanes<V>(Lv.nnz_ap)) {
      if constexpr (sizeof(V) == 4) {
        // FP32: eight lanes per A P block, then Q from the block's rows
        const float* Pb = Lv.p32;
        float* APb = Lv.ap32;
        float* Qb = Lv.q32;
        const float wl = (float)rho_f[1];
        const int lane = threadIdx.x & 31, r = lane & 7, gbase = lane & 24;
        const int stride = (gthreads >> 5) << 2, pos = ((gtid >> 5) << 2) + (lane >> 3);
        for (int k = 0; k * stride < Lv.nnz_ap; ++k) {
          const int bi = snake(k, stride, pos);
          const bool on = bi < Lv.nnz_ap && r < 7;
          const int b = bi < Lv.nnz_ap ? __ldg(Lv.ord2 + bi) : 0;
          float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          if (on) {
            recipe_row_f32(g, Lv, l, (float)lam, Lv.r2, __ldg(Lv.r2_ptr + b), __ldg(Lv.r2_ptr + b + 1), Pb, r, acc);
#pragma unroll
            for (int jj = 0; jj < 7; ++jj) APb[(size_t)b * BLK32 + r * 7 + jj] = acc[jj];
          }
          if (A.dense) {
            int u = 0, pb = -1;
            if (on) {
              u = __ldg(Lv.ap_row + b);
              pb = __ldg(Lv.ap_pblk + b);
            }
            const float* M = on ? (l == 0 ? g.minv32 : Lv.dinv32) + (size_t)u * BLK32 : nullptr;
            const float* Y = (on && pb >= 0) ? Pb + (size_t)pb * BLK32 : nullptr;
            float out[7];
            if (l == 0) smooth_row<true>(M, Y, wl, r, gbase, acc, out);
            else smooth_row<false>(M, Y, wl, r, gbase, acc, out);
            if (on)
#pragma unroll
              for (int jj = 0; jj < 7; ++jj) Qb[(size_t)b * BLK32 + r * 7 + jj] = out[jj];
          }
        }
      }
    } else {
      const int slot = threadIdx.x >> 6, t = threadIdx.x & 63;
      const int i = t / 7, j = t - 7 * (t / 7);
      const bool lane_on = t < 49;
      const V* Pb = AV<V>::p(Lv);
      V* APb = AV<V>::ap(Lv);
      const V* Dl = l == 0 ? AV<V>::minv(g) : AV<V>::dinv(Lv);
      V* Qb = AV<V>::q(Lv);
      const V wl = V(rho_f[1]);
      const int stride = gridDim.x * TEAMS, pos = blockIdx.x * TEAMS + slot;
      for (int k = 0; k * stride < Lv.nnz_ap; ++k) {
        const int bi = snake(k, stride, pos);
        if (bi >= Lv.nnz_ap) continue;
        const int b = __ldg(Lv.ord2t + bi);
        V drow[7], pv = V(0);
        if (A.dense && lane_on) {
          const int u = __ldg(Lv.ap_row + b), pb = __ldg(Lv.ap_pblk + b);
#pragma unroll
          for (int k = 0; k < 7; ++k) drow[k] = __ldg(Dl + (size_t)u * BLK + i * 7 + k);
          if (pb >= 0) pv = __ldcg(Pb + (size_t)pb * BLK + i * 7 + j);
        }
        if (lane_on) {
          const int e0 = __ldg(Lv.r2_ptr + b), e1 = __ldg(Lv.r2_ptr + b + 1);
          const V v = l == 0 ? recipe_ax<V, true>(g, nullptr, lam, Lv.r2, e0, e1, Pb, i, j)
                             : recipe_ax<V, false>(g, AV<V>::a(Lv), lam, Lv.r2, e0, e1, Pb, i, j);
          APb[(size_t)b * BLK + i * 7 + j] = v;
          sacc[slot][t] = v;
        }
        if (A.dense) {
          team_sync(slot);
          if (lane_on) {
            V sd = V(0);
#pragma unroll
            for (int k = 0; k < 7; ++k) sd += drow[k] * sacc[slot][k * 7 + j];
            Qb[(size_t)b * BLK + i * 7 + j] = pv - wl * sd;
          }
          team_sync(slot);
        }
      }
    }
    if (!grid_sync(counter, abort_flag, target)) goto timeout;
    if (lagged) break;   // the coarse levels of the last complete set-up stay
    // ---- A_next = P^T (A P), upper blocks ----
    if (fuse) {   // power step 3: y3 = D^-1 A y2 / |y2|
      const double2 nn = grid_norm_after_sync(partial + gridDim.x);
      const double ny2 = power_step<V>(g, Lv, l, lam, AV<V>::pw(A, 1), V(nn.y), AV<V>::pw(A, 0));
      block_partial(ny2, partial);
    }
    if (row_lanes<V>(Lv.nnz_next)) {
      if constexpr (sizeof(V) == 4) {
        // FP32: eight lanes per upper block of the next level, sum of P^T (A P)
        const float* Pb = Lv.p32;
        const float* APb = Lv.ap32;
        float* An = Ln.a32;
        const int lane = threadIdx.x & 31, r = lane & 7;
        const int stride = (gthreads >> 5) << 2, pos = ((gtid >> 5) << 2) + (lane >> 3);
        for (int k = 0; k * stride < Lv.nnz_next; ++k) {
          const int bi = snake(k, stride, pos);
          if (bi >= Lv.nnz_next || r >= 7) continue;
          const int b = __ldg(Lv.ord3 + bi);
          const int e0 = __ldg(Lv.r3_ptr + b), e1 = __ldg(Lv.r3_ptr + b + 1);
          if (e0 == e1) continue;   // mirrored block
          float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          for (int e = e0; e < e1; ++e) {
            const int2 t = __ldg(Lv.r3 + e);
            float X[52];
            ld_x52<false>(APb + (size_t)t.y * BLK32, X);
            mac_row<false, true>(Pb + (size_t)t.x * BLK32, r, X, acc);
          }
#pragma unroll
          for (int jj = 0; jj < 7; ++jj) An[(size_t)b * BLK32 + r * 7 + jj] = acc[jj];
        }
      }
    } else {
      const int slot = threadIdx.x >> 6, t = threadIdx.x & 63;
      const int i = t / 7, j = t - 7 * (t / 7);
      const V* Pb = AV<V>::p(Lv);
      const V* APb = AV<V>::ap(Lv);
      V* An = AV<V>::a(Ln);
      const int stride = gridDim.x * TEAMS, pos = blockIdx.x * TEAMS + slot;
      for (int k = 0; k * stride < Lv.nnz_next; ++k) {
        const int bi = snake(k, stride, pos);
        if (bi >= Lv.nnz_next || t >= 49) continue;
        const int b = __ldg(Lv.ord3 + bi);
        const int e0 = __ldg(Lv.r3_ptr + b), e1 = __ldg(Lv.r3_ptr + b + 1);
        if (e0 == e1) continue;   // mirrored block
        An[(size_t)b * BLK + i * 7 + j] = recipe_ptq<V>(Lv.r3, e0, e1, Pb, APb, i, j);
      }
    }
    if (!grid_sync(counter, abort_flag, target)) goto timeout;
    if (fuse) {   // the refined estimate |y3| and the vector for the next set-up
      const double2 nn = grid_norm_after_sync(partial);
      if (gtid == 0 && nn.x > 1e-30 && isfinite(nn.x)) A.rho_next[l] = nn.x;
      const V* y3 = AV<V>::pw(A, 0);
      for (int t = gtid; t < Lv.n * VEC; t += gthreads) pv[t] = __ldcg(y3 + t);
    }
    // ---- mirror the lower blocks, and the next level's D^-1 in the same
    // phase (it reads only diagonal blocks, which the products wrote; the
    // mirror writes only lower blocks) ----
    {
      V* An = AV<V>::a(Ln);
      for (int t = gtid; t < Lv.nnz_next * 49; t += gthreads) {
        const int b = t / 49, ij = t - 49 * b;
        const int src = __ldg(Ln.a_src + b);
        if (src < 0) continue;
        const int i = ij / 7, j = ij - 7 * (ij / 7);
        An[(size_t)b * BLK + i * 7 + j] = __ldcg(An + (size_t)src * BLK + j * 7 + i);
      }
    }
    if (l + 1 < A.L) {
      // one 64-thread team per node
      const V* An = AV<V>::a(Ln);
      const int slot = threadIdx.x >> 6, t = threadIdx.x & 63;
      for (int c0 = blockIdx.x * TEAMS; c0 < Ln.n; c0 += gridDim.x * TEAMS) {
        const int c = c0 + slot;
        const bool has = c < Ln.n;
        inv7_spd_team<V, true>(An + (size_t)(has ? __ldg(Ln.a_ptr + c) : 0) * BLK,
                               AV<V>::dinv(Ln) + (size_t)(has ? c : 0) * BLK, has, smat[slot], t);
      }
    }
    if (!grid_sync(counter, abort_flag, target)) goto timeout;
  }
  // ---- coarsest level: dense inverse (block 0, Gauss-Jordan on the SPD matrix) ----
  if (blockIdx.x == 0 && !lagged) {
    if (sizeof(V) == 4) coarsest_inverse_f32(A, reinterpret_cast<float*>(dense));
    else coarsest_inverse_f64(A, dense);
    if (threadIdx.x == 0) A.warm[warm_slot] = 1;
  }
  // ---- level L - 1: W = Q C^-1 Q^T, the coarse correction as one dense product ----
  // (a lagged set-up keeps the coarse levels, so W stays unless Q is the finest)
  if (A.dense && (!lagged || A.L == 1)) {
    const AmgLevel& Ld = A.lv[A.L - 1];
    const int nd = Ld.n, nL = A.nL;
    const V* Qb = AV<V>::q(Ld);
    const V* Ci = AV<V>::cinv(A);
    V* Hb = AV<V>::h(A);
    V* Wb = AV<V>::w(A);
    const int slot = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int i = t / 7, j = t - 7 * (t / 7);
    const bool lane_on = t < 49;
    if (!grid_sync(counter, abort_flag, target)) goto timeout;
    // H[u][c] = sum over the blocks k of row u of Q: Q_k C^-1[col k][c]
    for (int b = blockIdx.x * TEAMS + slot; b < nd * nL; b += gridDim.x * TEAMS) {
      if (!lane_on) continue;
      const int u = b / nL, c = b - nL * u;
      V acc = V(0);
      for (int k = __ldg(Ld.ap_ptr + u); k < __ldg(Ld.ap_ptr + u + 1); ++k) {
        const V* qk = Qb + (size_t)k * BLK + i * 7;
        const V* ck = Ci + ((size_t)__ldg(Ld.ap_col + k) * nL + c) * BLK + j;
#pragma unroll
        for (int m = 0; m < 7; ++m) acc += __ldcg(qk + m) * __ldcg(ck + m * 7);
      }
      Hb[(size_t)b * BLK + i * 7 + j] = acc;
    }
    if (!grid_sync(counter, abort_flag, target)) goto timeout;
    // W[u][v] = sum over the blocks k of row v of Q: H[u][col k] Q_k^T
    for (int b = blockIdx.x * TEAMS + slot; b < nd * nd; b += gridDim.x * TEAMS) {
      if (!lane_on) continue;
      const int u = b / nd, v = b - nd * u;
      V acc = V(0);
      for (int k = __ldg(Ld.ap_ptr + v); k < __ldg(Ld.ap_ptr + v + 1); ++k) {
        const V* hk = Hb + ((size_t)u * nL + __ldg(Ld.ap_col + k)) * BLK + i * 7;
        const V* qk = Qb + (size_t)k * BLK + j * 7;
#pragma unroll
        for (int m = 0; m < 7; ++m) acc += __ldcg(hk + m) * __ldcg(qk + m);
      }
      Wb[(size_t)b * BLK + i * 7 + j] = acc;
    }
  }
  grid_sync_release(&st->ticket[T_AMG_DONE], counter, nullptr);
  return;
timeout:
  // a barrier wait ran out: stop the solve and report a device failure
  // (every block that gave up writes the same values: block 0 may be the absent one)
  if (threadIdx.x == 0) {
    st->status = PGO_ERR_CUDA;
    st->stop_reason = 4;
    st->done = 1;
  }
}

static int amg_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

cudaError_t launch_amg_setup(const DevGraph& g, const AmgDev& amg, int mixed, int lm, cudaStream_t s) {
  const int blocks = amg_sms();
  const size_t n7 = (size_t)7 * amg.nL;
  // block 0: the coarsest operator twice (double-buffered elimination) and a scale vector
  const size_t smem = (2 * n7 * n7 + n7) * sizeof(double);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(mixed ? SetupShape<float>::THREADS : SetupShape<double>::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (mixed) {
    cudaError_t e = cudaFuncSetAttribute(k_amg_setup<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k_amg_setup<float>, g, lm);
  }
  cudaError_t e = cudaFuncSetAttribute(k_amg_setup<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, k_amg_setup<double>, g, lm);
}

// Test hook: the grid-barrier wait limit of this file's kernels (0: 2 s).
void set_barrier_limit_amg(unsigned long long ns) {
  cudaMemcpyToSymbol(g_barrier_limit_ns, &ns, sizeof(ns));
  cudaGetLastError();
}

}  // namespace pgo
