// Branch and bound for the QAP with RLT2 dual-ascent bounds on one GPU
// (Section 4): polytomic branching on the facilities in a fixed placement order
// (rules 1-3), a best-first heap of open nodes (deeper nodes first among equal
// bounds, the BstFS + DFS hybrid), parent -> child multiplier warm starts for
// parents up to a depth limit, and early termination of each node's ascent
// (min-gap against the incumbent, the stall rule of the parameters).
//
// The driver is a client of the library's own C ABI (include/rlt2.h): every
// node is a context bounded by the same kernels as a single dual ascent;
// children of a kept parent are derived on the device from its multiplier-
// adjusted costs (rlt2_create_child).  Host work is the heap, the placement
// order and the enumeration of nodes with at most two free facilities.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <queue>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "rlt2.h"
#include "rlt2_internal.h"

namespace {

struct Node {
  double lb;
  int depth;                 // facilities fixed (the first `depth` of the placement order)
  std::vector<int> partial;  // n entries, location or -1
  rlt2_ctx* state;           // the node's bounded context, kept to warm-start its children (or nullptr)
  long long seq;             // creation order
};

struct Worse {
  // priority: smaller bound first; among equal bounds the deeper node, then the newer one
  bool operator()(const Node* a, const Node* b) const {
    if (a->lb != b->lb) return a->lb > b->lb;
    if (a->depth != b->depth) return a->depth < b->depth;
    return a->seq < b->seq;
  }
};

// Placement order of the facilities (Section 4): rule 1 = index order; rule 2
// (3) = start with the largest (smallest) total interaction sum_j f_ij + f_ji,
// then repeatedly the free facility with the largest (smallest) interaction
// with the facilities already placed; ties to the lower index.
std::vector<int> placement_order(int n, const double* F, int rule) {
  std::vector<int> order;
  if (rule == 1) {
    for (int i = 0; i < n; ++i) order.push_back(i);
    return order;
  }
  const bool largest = rule == 2;
  std::vector<char> used(n, 0);
  std::vector<double> score(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (j != i) score[i] += F[i * n + j] + F[j * n + i];
  for (int step = 0; step < n; ++step) {
    int pick = -1;
    for (int i = 0; i < n; ++i) {
      if (used[i]) continue;
      if (pick < 0 || (largest ? score[i] > score[pick] : score[i] < score[pick])) pick = i;
    }
    used[pick] = 1;
    order.push_back(pick);
    // from now on the score is the interaction with the placed facilities
    if (step == 0) std::fill(score.begin(), score.end(), 0.0);
    for (int i = 0; i < n; ++i)
      if (!used[i]) score[i] += F[i * n + pick] + F[pick * n + i];
  }
  return order;
}

double qap_value(int n, const double* F, const double* D, const double* B, const std::vector<int>& s) {
  double v = 0.0;
  for (int i = 0; i < n; ++i) {
    if (B) v += B[i * n + s[i]];
    for (int j = 0; j < n; ++j) v += F[i * n + j] * D[s[i] * n + s[j]];
  }
  return v;
}

bool integral(const double* x, size_t k) {
  for (size_t i = 0; i < k; ++i)
    if (x[i] != std::floor(x[i]) || std::fabs(x[i]) > 1e15) return false;
  return true;
}

}  // namespace

extern "C" void rlt2_bnb_options_default(rlt2_bnb_options* o) {
  if (!o) return;
  o->order_rule = 3;
  o->iters_root = 200;
  o->iters_node = 100;
  o->warm_depth = 64;
  o->max_states = 4096;
  o->max_nodes = 0;
  o->time_limit_s = 0.0;
  o->ub0 = 0.0;
  o->abs_tol = -1.0;
  o->max_state_bytes = 0.0;
  o->batch_children = 1;
}

extern "C" rlt2_status rlt2_bnb_solve(int n, const double* F, const double* D, const double* B, const rlt2_params* p,
                                      const rlt2_bnb_options* opt, double* best, int* perm, double* root_lb,
                                      long long* stats, void* stream) {
  if (n < 3 || n > 64 || !F || !D || !best || !perm) {
    rlt2::set_error("rlt2_bnb_solve: need 3 <= n <= 64 and non-NULL F, D, best, perm");
    return RLT2_EINVAL;
  }
  rlt2_bnb_options o;
  rlt2_bnb_options_default(&o);
  if (opt) o = *opt;
  if (o.order_rule < 1 || o.order_rule > 3 || o.iters_root < 1 || o.iters_node < 1 || o.max_states < 0 ||
      o.max_nodes < 0 || !std::isfinite(o.time_limit_s) || !std::isfinite(o.ub0) || !std::isfinite(o.abs_tol) ||
      !(o.max_state_bytes >= 0.0) || (o.batch_children != 0 && o.batch_children != 1)) {
    rlt2::set_error("rlt2_bnb_solve: options out of range");
    return RLT2_EINVAL;
  }
  double state_budget = o.max_state_bytes;
  if (state_budget <= 0.0) {
    size_t fr = 0, tot = 0;
    const cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return rlt2::cuda_fail(e, "rlt2_bnb_solve: cudaMemGetInfo");
    state_budget = 0.5 * (double)fr;
  }
  rlt2_params prm;
  rlt2_params_default(&prm);
  if (p) prm = *p;
  if (prm.variant != 0) {  // children inherit the S variant's multiplier-adjusted costs
    rlt2::set_error("rlt2_bnb_solve: node parameters must select the S variant");
    return RLT2_EINVAL;
  }
  const size_t nn = (size_t)n * n;
  const bool whole = integral(F, nn) && integral(D, nn) && (!B || integral(B, nn));
  const auto t_start = std::chrono::steady_clock::now();
  const std::vector<int> order = placement_order(n, F, o.order_rule);

  double inc = o.ub0 > 0.0 ? o.ub0 : INFINITY;
  std::vector<int> inc_perm;
  long long bounded = 0, branched = 0, leaves = 0, iterations = 0, warm = 0, cold = 0;
  int max_depth = 0, kept = 0;
  double kept_bytes = 0.0;
  // device bytes of a context with residual size r (z array, tile arrays, duals)
  auto ctx_bytes = [](int r) {
    const double T = (double)r * r * (r - 1) * (r - 1);
    return 8.0 * (T * (r - 2) * (r - 2) + 6.0 * T + 2.0 * T * (r - 2)) + (1 << 20);
  };
  bool limited = false;
  rlt2_status st = RLT2_OK;
  auto tol = [&]() { return o.abs_tol >= 0.0 ? o.abs_tol : (whole ? 1.0 - 1e-6 : 1e-9 * std::max(1.0, std::fabs(inc))); };
  auto fathomed = [&](double lb) { return std::isfinite(inc) && lb >= inc - tol(); };
  auto offer = [&](double v, const std::vector<int>& s) {
    if (v < inc) {
      inc = v;
      inc_perm = s;
    }
  };
  // node parameters: stop the ascent once the node is fathomed (min-gap against the incumbent)
  auto node_params = [&]() {
    rlt2_params q = prm;
    if (std::isfinite(inc)) {
      q.ub = inc;
      q.min_gap = tol() / std::max(1e-300, std::fabs(inc));
    }
    return q;
  };
  // a bounded node context: read its bound and offer its X-LAP primal
  auto harvest = [&](rlt2_ctx* c, int done, double* lb_out) -> rlt2_status {
    double lb = 0.0, blb = 0.0, ub = 0.0;
    int its = 0;
    std::vector<int> up(n);
    rlt2_status s = rlt2_bound(c, &lb, &blb, &ub, nullptr, up.data(), &its);
    if (s != RLT2_OK) return s;
    ++bounded;
    iterations += done;
    if (std::isfinite(ub)) offer(qap_value(n, F, D, B, up), up);
    *lb_out = blb;
    return RLT2_OK;
  };
  // bound one node context: iterate, read the bound and its X-LAP primal
  auto bound = [&](rlt2_ctx* c, int iters, double* lb_out) -> rlt2_status {
    int done = 0;
    rlt2_status s = rlt2_iterate(c, iters, nullptr, &done);
    if (s != RLT2_OK) return s;
    return harvest(c, done, lb_out);
  };
  const bool batched = o.batch_children == 1 && !prm.half_z && prm.warm != 2;
  // nodes with at most two free facilities: enumerate their completions
  auto enumerate = [&](const std::vector<int>& part) {
    std::vector<int> ff, fl;
    std::vector<char> used(n, 0);
    for (int i = 0; i < n; ++i)
      if (part[i] >= 0) used[part[i]] = 1;
    for (int i = 0; i < n; ++i)
      if (part[i] < 0) ff.push_back(i);
    for (int q = 0; q < n; ++q)
      if (!used[q]) fl.push_back(q);
    std::sort(fl.begin(), fl.end());
    do {
      std::vector<int> s = part;
      for (size_t a = 0; a < ff.size(); ++a) s[ff[a]] = fl[a];
      offer(qap_value(n, F, D, B, s), s);
      ++leaves;
    } while (std::next_permutation(fl.begin(), fl.end()));
  };

  std::priority_queue<Node*, std::vector<Node*>, Worse> heap;
  long long seq = 0;
  double rlb = -INFINITY;
  {
    rlt2_params q = node_params();
    rlt2_ctx* root = nullptr;
    if ((st = rlt2_create(n, F, D, B, nullptr, &q, stream, &root)) != RLT2_OK) return st;
    if ((st = bound(root, o.iters_root, &rlb)) != RLT2_OK) {
      rlt2_destroy(root);
      return st;
    }
    Node* nd = new Node{rlb, 0, std::vector<int>(n, -1), nullptr, seq++};
    if (o.warm_depth >= 0 && o.max_states > 0 && ctx_bytes(n) <= state_budget) {
      nd->state = root;
      ++kept;
      kept_bytes += ctx_bytes(n);
    } else {
      rlt2_destroy(root);
    }
    heap.push(nd);
  }
  while (!heap.empty()) {
    Node* nd = heap.top();
    heap.pop();
    if (fathomed(nd->lb) || limited) {
      if (!fathomed(nd->lb)) limited = true;
      if (nd->state) {
        rlt2_destroy(nd->state);
        --kept;
        kept_bytes -= ctx_bytes(n - nd->depth);
      }
      delete nd;
      continue;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if ((o.max_nodes > 0 && bounded >= o.max_nodes) || (o.time_limit_s > 0.0 && secs > o.time_limit_s)) {
      limited = true;
      heap.push(nd);
      continue;
    }
    // branch: the next facility of the order at every free location
    const int fac = order[nd->depth];
    std::vector<char> used(n, 0);
    for (int i = 0; i < n; ++i)
      if (nd->partial[i] >= 0) used[nd->partial[i]] = 1;
    ++branched;
    const int depth = nd->depth + 1;
    max_depth = std::max(max_depth, depth);
    // a bounded child: fathomed, or pushed on the heap (its context kept for
    // its own children within the depth and memory limits)
    auto place = [&](rlt2_ctx* c, const std::vector<int>& part, double lb) {
      if (fathomed(lb)) {
        rlt2_destroy(c);
        return;
      }
      Node* ch = new Node{lb, depth, part, nullptr, seq++};
      if (depth <= o.warm_depth && kept < o.max_states && kept_bytes + ctx_bytes(n - depth) <= state_budget) {
        ch->state = c;
        ++kept;
        kept_bytes += ctx_bytes(n - depth);
      } else {
        rlt2_destroy(c);
      }
      heap.push(ch);
    };
    std::vector<rlt2_ctx*> kids;  // batched: created first, then bounded together
    std::vector<std::vector<int>> kparts;
    for (int loc = 0; loc < n && st == RLT2_OK; ++loc) {
      if (used[loc]) continue;
      std::vector<int> part = nd->partial;
      part[fac] = loc;
      if (n - depth <= 2) {
        enumerate(part);
        continue;
      }
      rlt2_params q = node_params();
      rlt2_ctx* c = nullptr;
      if (nd->state) {
        st = rlt2_create_child(nd->state, fac, loc, &q, &c);
        ++warm;
      } else {
        st = rlt2_create(n, F, D, B, part.data(), &q, stream, &c);
        ++cold;
      }
      if (st != RLT2_OK) break;
      if (batched) {
        kids.push_back(c);
        kparts.push_back(part);
        continue;
      }
      // one at a time: each child is bounded before the next is created
      double lb = -INFINITY;
      if ((st = bound(c, o.iters_node, &lb)) != RLT2_OK) {
        rlt2_destroy(c);
        break;
      }
      place(c, part, lb);
    }
    if (!kids.empty()) {
      std::vector<int> done(kids.size(), 0);
      std::vector<double> klb(kids.size(), -INFINITY);
      if (st == RLT2_OK) st = rlt2_iterate_many(kids.data(), (int)kids.size(), o.iters_node, done.data());
      for (size_t k = 0; k < kids.size() && st == RLT2_OK; ++k) st = harvest(kids[k], done[k], &klb[k]);
      for (size_t k = 0; k < kids.size(); ++k) {
        if (st != RLT2_OK) rlt2_destroy(kids[k]);
        else place(kids[k], kparts[k], klb[k]);
      }
    }
    if (nd->state) {
      rlt2_destroy(nd->state);
      --kept;
      kept_bytes -= ctx_bytes(n - nd->depth);
    }
    delete nd;
    if (st != RLT2_OK) break;
  }
  while (!heap.empty()) {
    Node* nd = heap.top();
    heap.pop();
    if (nd->state) rlt2_destroy(nd->state);
    delete nd;
  }
  if (st != RLT2_OK) return st;
  *best = inc;
  for (int i = 0; i < n; ++i) perm[i] = inc_perm.empty() ? -1 : inc_perm[i];
  if (root_lb) *root_lb = rlb;
  if (stats) {
    stats[0] = bounded;
    stats[1] = branched;
    stats[2] = leaves;
    stats[3] = iterations;
    stats[4] = max_depth;
    stats[5] = (!limited && !inc_perm.empty()) ? 1 : 0;
    stats[6] = warm;
    stats[7] = cold;
  }
  return RLT2_OK;
}
