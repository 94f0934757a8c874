// bvh_build.cpp — multi-threaded binned-SAH BVH2 builder.
//
// The paper builds its BVH with binned SAH (Sec. 4) and notes that the
// culling does not depend on the branching factor or the builder.  This
// builder follows one canonical rule set so that its tree is fully
// determined by the triangles (and therefore reproducible by an independent
// sequential implementation):
//   * triangle box = float min/max of its vertices, centroid (double) =
//     0.5 * (lo + hi);
//   * a range of n <= max_leaf triangles becomes a leaf;
//   * else, per axis whose centroid extent is > 0: bin = min(bins-1,
//     (int)((c - cmin) * (bins / extent))); the plane between bins i and
//     i+1 costs SA(left)*|left| + SA(right)*|right| (the greedy form of
//     Eq. 1, double); the cheapest plane with both sides non-empty wins,
//     ties to the lower axis, then the lower plane;
//   * no valid plane (all centroids equal): the first n/2 go left;
//   * stable partition; nodes numbered in pre-order.
// Float min/max, integer counts and the fixed cost expression make every
// decision independent of how the work is split across threads.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>

#include "internal.h"

namespace sc {
namespace {

struct TriRec {
  float lo[3], hi[3];
  double c[3];
};

struct Ref {
  int kind;  // 0 leaf (a = first position, b = count), 1 top node (a), 2 task node (a = task, b = local)
  int32_t a, b;
};

struct BNode {
  Ref ch[2];
  float box[2][6];
};

inline void box_empty(float* b) {
  b[0] = b[1] = b[2] = INFINITY;
  b[3] = b[4] = b[5] = -INFINITY;
}
inline void box_grow(float* b, const float* lo, const float* hi) {
  for (int k = 0; k < 3; ++k) {
    b[k] = std::fmin(b[k], lo[k]);
    b[3 + k] = std::fmax(b[3 + k], hi[k]);
  }
}
inline double area(const float* b) {
  double dx = (double)b[3] - (double)b[0];
  double dy = (double)b[4] - (double)b[1];
  double dz = (double)b[5] - (double)b[2];
  return 2.0 * ((dx * dy + dy * dz) + dz * dx);
}
inline int bin_index(double c, double cmin, double ext, int nb) {
  int i = (int)((c - cmin) * ((double)nb / ext));
  if (i > nb - 1) i = nb - 1;
  if (i < 0) i = 0;
  return i;
}

constexpr int kMaxBins = 256;

struct Bins {
  int64_t cnt[3][kMaxBins];
  float box[3][kMaxBins][6];
  void clear(int nb) {
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < nb; ++i) {
        cnt[k][i] = 0;
        box_empty(box[k][i]);
      }
  }
  void merge(const Bins& o, int nb) {
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < nb; ++i) {
        cnt[k][i] += o.cnt[k][i];
        box_grow(box[k][i], o.box[k][i], o.box[k][i] + 3);
      }
  }
};

struct Ctx {
  const TriRec* rec;
  int32_t* perm;
  int32_t* tmp;
  int max_leaf, nb, threads;
  int64_t par_min;  // ranges at least this large use threads inside
};

// Range statistics: box, centroid bounds.
void range_stats(const Ctx& x, int64_t begin, int64_t end, bool par, float* box,
                 double* cmin, double* cmax) {
  auto body = [&](int64_t b, int64_t e, float* bx, double* mn, double* mx) {
    box_empty(bx);
    for (int k = 0; k < 3; ++k) {
      mn[k] = INFINITY;
      mx[k] = -INFINITY;
    }
    for (int64_t i = b; i < e; ++i) {
      const TriRec& t = x.rec[x.perm[i]];
      box_grow(bx, t.lo, t.hi);
      for (int k = 0; k < 3; ++k) {
        mn[k] = t.c[k] < mn[k] ? t.c[k] : mn[k];
        mx[k] = t.c[k] > mx[k] ? t.c[k] : mx[k];
      }
    }
  };
  if (!par) {
    body(begin, end, box, cmin, cmax);
    return;
  }
  int P = x.threads;
  std::vector<float> pb(6 * P);
  std::vector<double> pmn(3 * P), pmx(3 * P);
  int64_t n = end - begin;
  parallel_ranges(n, P, [&](int64_t b, int64_t e, int p) {
    body(begin + b, begin + e, &pb[6 * p], &pmn[3 * p], &pmx[3 * p]);
  });
  box_empty(box);
  for (int k = 0; k < 3; ++k) {
    cmin[k] = INFINITY;
    cmax[k] = -INFINITY;
  }
  for (int p = 0; p < P; ++p) {
    box_grow(box, &pb[6 * p], &pb[6 * p + 3]);
    for (int k = 0; k < 3; ++k) {
      cmin[k] = pmn[3 * p + k] < cmin[k] ? pmn[3 * p + k] : cmin[k];
      cmax[k] = pmx[3 * p + k] > cmax[k] ? pmx[3 * p + k] : cmax[k];
    }
  }
}

// Chooses the split of perm[begin, end) and partitions it; returns mid.
int64_t split(const Ctx& x, int64_t begin, int64_t end, bool par, const double* cmin,
              const double* cmax) {
  const int nb = x.nb;
  double ext[3];
  bool use[3];
  for (int k = 0; k < 3; ++k) {
    ext[k] = cmax[k] - cmin[k];
    use[k] = ext[k] > 0.0;
  }
  auto bin_range = [&](int64_t b, int64_t e, Bins& bins) {
    bins.clear(nb);
    for (int64_t i = b; i < e; ++i) {
      const TriRec& t = x.rec[x.perm[i]];
      for (int k = 0; k < 3; ++k) {
        if (!use[k]) continue;
        int bi = bin_index(t.c[k], cmin[k], ext[k], nb);
        bins.cnt[k][bi] += 1;
        box_grow(bins.box[k][bi], t.lo, t.hi);
      }
    }
  };
  std::unique_ptr<Bins> bins(new Bins);
  int64_t n = end - begin;
  if (!par) {
    bin_range(begin, end, *bins);
  } else {
    int P = x.threads;
    std::vector<std::unique_ptr<Bins>> part(P);
    for (auto& p : part) p.reset(new Bins);
    parallel_ranges(n, P, [&](int64_t b, int64_t e, int p) {
      bin_range(begin + b, begin + e, *part[p]);
    });
    bins->clear(nb);
    for (int p = 0; p < P; ++p) bins->merge(*part[p], nb);
  }
  int best_axis = -1, best_plane = -1;
  double best_cost = INFINITY;
  for (int k = 0; k < 3; ++k) {
    if (!use[k]) continue;
    int64_t lc[kMaxBins], rc[kMaxBins];
    double la[kMaxBins], ra[kMaxBins];
    float acc[6];
    box_empty(acc);
    int64_t a = 0;
    for (int i = 0; i < nb - 1; ++i) {
      a += bins->cnt[k][i];
      box_grow(acc, bins->box[k][i], bins->box[k][i] + 3);
      lc[i] = a;
      la[i] = a > 0 ? area(acc) : 0.0;
    }
    box_empty(acc);
    a = 0;
    for (int i = nb - 1; i >= 1; --i) {
      a += bins->cnt[k][i];
      box_grow(acc, bins->box[k][i], bins->box[k][i] + 3);
      rc[i - 1] = a;
      ra[i - 1] = a > 0 ? area(acc) : 0.0;
    }
    for (int p = 0; p < nb - 1; ++p) {
      if (lc[p] == 0 || rc[p] == 0) continue;
      double cost = la[p] * (double)lc[p] + ra[p] * (double)rc[p];
      if (cost < best_cost) {
        best_cost = cost;
        best_axis = k;
        best_plane = p;
      }
    }
  }
  if (best_axis < 0) return begin + n / 2;
  const int ax = best_axis, pl = best_plane;
  const double cm = cmin[ax], ex = ext[ax];
  auto goes_left = [&](int32_t t) { return bin_index(x.rec[t].c[ax], cm, ex, nb) <= pl; };
  if (!par) {
    int64_t nl = 0, nr = 0;
    for (int64_t i = begin; i < end; ++i) {
      int32_t t = x.perm[i];
      if (goes_left(t)) x.perm[begin + nl++] = t;
      else x.tmp[begin + nr++] = t;
    }
    std::memcpy(x.perm + begin + nl, x.tmp + begin, sizeof(int32_t) * (size_t)nr);
    return begin + nl;
  }
  // parallel stable partition: count per part, then scatter to tmp
  int P = x.threads;
  std::vector<int64_t> left(P, 0), total(P, 0);
  parallel_ranges(n, P, [&](int64_t b, int64_t e, int p) {
    int64_t c = 0;
    for (int64_t i = begin + b; i < begin + e; ++i) c += goes_left(x.perm[i]);
    left[p] = c;
    total[p] = e - b;
  });
  std::vector<int64_t> loff(P), roff(P);
  int64_t nl = 0;
  for (int p = 0; p < P; ++p) nl += left[p];
  int64_t l = 0, r = nl;
  for (int p = 0; p < P; ++p) {
    loff[p] = l;
    roff[p] = r;
    l += left[p];
    r += total[p] - left[p];
  }
  parallel_ranges(n, P, [&](int64_t b, int64_t e, int p) {
    int64_t li = loff[p], ri = roff[p];
    for (int64_t i = begin + b; i < begin + e; ++i) {
      int32_t t = x.perm[i];
      if (goes_left(t)) x.tmp[begin + li++] = t;
      else x.tmp[begin + ri++] = t;
    }
  });
  parallel_ranges(n, P, [&](int64_t b, int64_t e, int) {
    std::memcpy(x.perm + begin + b, x.tmp + begin + b, sizeof(int32_t) * (size_t)(e - b));
  });
  return begin + nl;
}

struct Task {
  int64_t begin, end;
  int depth;
  std::vector<BNode> nodes;
  int max_depth = 0;
};

struct Builder {
  Ctx x;
  std::vector<BNode> top;
  std::vector<Task> tasks;
  int64_t task_max;
  int max_depth = 0;

  // Sequential recursive build inside a task (local pre-order).
  Ref build_seq(Task& t, int64_t begin, int64_t end, int depth, float* box) {
    double cmin[3], cmax[3];
    range_stats(x, begin, end, false, box, cmin, cmax);
    if (depth > t.max_depth) t.max_depth = depth;
    int64_t n = end - begin;
    if (n <= x.max_leaf) return Ref{0, (int32_t)begin, (int32_t)n};
    int64_t mid = split(x, begin, end, false, cmin, cmax);
    int32_t id = (int32_t)t.nodes.size();
    t.nodes.emplace_back();
    float b0[6], b1[6];
    Ref r0 = build_seq(t, begin, mid, depth + 1, b0);
    Ref r1 = build_seq(t, mid, end, depth + 1, b1);
    BNode& nd = t.nodes[id];
    nd.ch[0] = r0;
    nd.ch[1] = r1;
    std::memcpy(nd.box[0], b0, sizeof(b0));
    std::memcpy(nd.box[1], b1, sizeof(b1));
    return Ref{2, -1, id};  // task index patched by the caller
  }

  // Top levels: threads inside each split; small ranges become tasks.
  Ref build_top(int64_t begin, int64_t end, int depth, float* box) {
    int64_t n = end - begin;
    bool par = n >= x.par_min;
    double cmin[3], cmax[3];
    range_stats(x, begin, end, par, box, cmin, cmax);
    if (depth > max_depth) max_depth = depth;
    if (n <= x.max_leaf) return Ref{0, (int32_t)begin, (int32_t)n};
    if (n <= task_max) {
      Task t;
      t.begin = begin;
      t.end = end;
      t.depth = depth;
      tasks.push_back(std::move(t));
      return Ref{2, (int32_t)(tasks.size() - 1), 0};
    }
    int64_t mid = split(x, begin, end, par, cmin, cmax);
    int32_t id = (int32_t)top.size();
    top.emplace_back();
    float b0[6], b1[6];
    Ref r0 = build_top(begin, mid, depth + 1, b0);
    Ref r1 = build_top(mid, end, depth + 1, b1);
    BNode& nd = top[id];
    nd.ch[0] = r0;
    nd.ch[1] = r1;
    std::memcpy(nd.box[0], b0, sizeof(b0));
    std::memcpy(nd.box[1], b1, sizeof(b1));
    return Ref{1, id, 0};
  }
};

}  // namespace

void build_bvh(Bvh& b, const float* tris, int64_t n, int max_leaf, int bins,
               int threads) {
  double t0 = now_ms();
  b.ntri = n;
  b.tris.assign(tris, tris + 9 * n);
  b.perm.resize((size_t)n);
  std::vector<TriRec> rec((size_t)n);
  parallel_for(n, threads, 65536, [&](int64_t i) {
    const float* t = tris + 9 * i;
    for (int k = 0; k < 3; ++k) {
      rec[i].lo[k] = std::fmin(std::fmin(t[k], t[3 + k]), t[6 + k]);
      rec[i].hi[k] = std::fmax(std::fmax(t[k], t[3 + k]), t[6 + k]);
      rec[i].c[k] = 0.5 * ((double)rec[i].lo[k] + (double)rec[i].hi[k]);
    }
    b.perm[i] = (int32_t)i;
  });
  b.child.clear();
  b.count.clear();
  b.box.clear();
  b.ndepth.clear();
  b.nn = 0;
  b.max_depth = 0;
  if (n == 0) {
    b.root_child = -1;
    b.root_count = 0;
    box_empty(b.root_box);
    b.ms_bvh = now_ms() - t0;
    return;
  }
  std::vector<int32_t> tmp((size_t)n);
  Builder B;
  B.x = Ctx{rec.data(), b.perm.data(), tmp.data(), max_leaf, bins, threads, 1 << 18};
  B.task_max = std::max<int64_t>(4096, n / (int64_t)(threads * 16));
  if (threads <= 1) B.task_max = n;  // one task: plain sequential recursion
  Ref root = B.build_top(0, n, 0, b.root_box);
  // run the tasks (each a sequential subtree build on a disjoint range)
  parallel_for((int64_t)B.tasks.size(), threads, 1, [&](int64_t i) {
    Task& t = B.tasks[i];
    float bx[6];
    B.build_seq(t, t.begin, t.end, t.depth, bx);
  });
  for (auto& t : B.tasks) B.max_depth = std::max(B.max_depth, t.max_depth);
  b.max_depth = B.max_depth;
  // pre-order numbering
  int64_t total = (int64_t)B.top.size();
  for (auto& t : B.tasks) total += (int64_t)t.nodes.size();
  b.nn = total;
  b.child.resize(2 * total);
  b.count.resize(2 * total);
  b.box.resize(12 * total);
  b.ndepth.resize(total);
  struct Item {
    Ref r;
    int task;    // task that owns a local ref (kind 2 with b >= 0 inside a task)
    int depth;
    int64_t parent_slot;  // index into child/count to patch, -1 for root
  };
  auto node_of = [&](const Ref& r, int task) -> const BNode* {
    if (r.kind == 1) return &B.top[r.a];
    return &B.tasks[task].nodes[r.b];
  };
  int64_t next = 0;
  std::vector<Item> stack;
  // resolve the root slot
  auto resolve = [&](Ref r, int task, int& out_task) -> Ref {
    // a task's root is local node 0
    if (r.kind == 2 && r.a >= 0 && task < 0) {
      out_task = r.a;
      return Ref{2, r.a, 0};
    }
    out_task = task;
    return r;
  };
  {
    int tk;
    Ref r = resolve(root, -1, tk);
    if (r.kind == 0) {
      b.root_child = r.a;
      b.root_count = r.b;
    } else {
      b.root_child = 0;
      b.root_count = 0;
      stack.push_back(Item{r, tk, 0, -1});
    }
  }
  while (!stack.empty()) {
    Item it = stack.back();
    stack.pop_back();
    int64_t id = next++;
    if (it.parent_slot >= 0) b.child[it.parent_slot] = (int32_t)id;
    const BNode* nd = node_of(it.r, it.task);
    b.ndepth[id] = it.depth;
    for (int c = 0; c < 2; ++c) std::memcpy(&b.box[12 * id + 6 * c], nd->box[c], 24);
    // push right first so that the left subtree is numbered next
    for (int c = 1; c >= 0; --c) {
      Ref ch = nd->ch[c];
      int tk = it.task;
      if (ch.kind == 2 && it.r.kind == 1) {
        // reference from a top node to a task root
        tk = ch.a;
        ch = Ref{2, ch.a, 0};
      }
      if (ch.kind == 0) {
        b.child[2 * id + c] = ch.a;
        b.count[2 * id + c] = ch.b;
      } else {
        b.count[2 * id + c] = 0;
        stack.push_back(Item{ch, tk, it.depth + 1, 2 * id + c});
      }
    }
  }
  b.ms_bvh = now_ms() - t0;
}

double scene_eps(const float* tris, int64_t n, double eps_rel) {
  double s = 1.0;
  for (int64_t i = 0; i < 9 * n; ++i) {
    double a = std::fabs((double)tris[i]);
    if (a > s) s = a;
  }
  return eps_rel * s;
}

}  // namespace sc
