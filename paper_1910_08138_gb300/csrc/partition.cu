// partition.cu -- sub-block construction (Sec. 5.2): the cameras are split
// into sub-blocks by partitioning the visibility graph, balancing the
// estimated work and keeping the tie points few.
//
// Graph: one node per camera; two cameras are adjacent when they observe a
// common point, the edge weight being the number of such points. Node weight
// (the paper's empirical choice): the cube root of the sum, over the points
// the camera sees, of their observation counts.
//
// Partitioner (written here, in place of METIS): recursive bisection. A
// bisection grows one side from a pseudo-peripheral camera by breadth-first
// search (neighbours taken in order of their connection to the grown side)
// until it holds its share of the weight, then improves the cut by
// Fiduccia-Mattheyses passes (single moves of boundary cameras by gain, each
// side within 2 % of its share, each pass rolled back to its best prefix). k parts split
// into floor(k/2) and ceil(k/2) with weight shares in that ratio.
//
// Host code only: no GPU is used.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <queue>
#include <set>
#include <vector>

#include "../../include/rpba.h"

namespace {

struct Graph {
  int n = 0;
  std::vector<int> ptr, adj;  // CSR
  std::vector<double> ew;     // edge weights (shared points)
  std::vector<double> nw;     // node weights
};

// the node farthest (in hops) from start within the subset, by BFS
int farthest(const Graph &g, const std::vector<char> &in, int start, std::vector<int> &dist) {
  std::queue<int> q;
  dist[start] = 0;
  q.push(start);
  int last = start;
  std::vector<int> seen{start};
  while (!q.empty()) {
    int u = q.front();
    q.pop();
    last = u;
    for (int e = g.ptr[u]; e < g.ptr[u + 1]; e++) {
      int v = g.adj[e];
      if (!in[v] || dist[v] >= 0) continue;
      dist[v] = dist[u] + 1;
      seen.push_back(v);
      q.push(v);
    }
  }
  for (int u : seen) dist[u] = -1;
  return last;
}

// bisect `nodes` so that side 0 holds about `share` of their weight
void bisect(const Graph &g, const std::vector<int> &nodes, std::vector<char> &in, double share,
            std::vector<int> &side, std::vector<int> &dist) {
  double W = 0.0;
  for (int u : nodes) W += g.nw[u];
  double target = share * W;
  for (int u : nodes) side[u] = 1;
  // grow side 0 from a pseudo-peripheral node, covering every connected piece
  std::vector<char> grown(g.n, 0);
  double w0 = 0.0;
  size_t next_seed = 0;
  while (w0 < target) {
    while (next_seed < nodes.size() && grown[nodes[next_seed]]) next_seed++;
    if (next_seed >= nodes.size()) break;
    int start = farthest(g, in, farthest(g, in, nodes[next_seed], dist), dist);
    if (grown[start]) start = nodes[next_seed];
    // priority: connection weight to the grown side (max first), then id
    std::priority_queue<std::pair<double, int>> pq;
    std::map<int, double> conn;
    pq.push({0.0, -start});
    while (!pq.empty() && w0 < target) {
      auto [c, mu] = pq.top();
      pq.pop();
      int u = -mu;
      if (grown[u]) continue;
      if (conn.count(u) && conn[u] > c) continue;  // a stale entry
      grown[u] = 1;
      side[u] = 0;
      w0 += g.nw[u];
      for (int e = g.ptr[u]; e < g.ptr[u + 1]; e++) {
        int v = g.adj[e];
        if (!in[v] || grown[v]) continue;
        double cv = (conn[v] += g.ew[e]);
        pq.push({cv, -v});
      }
    }
  }
  // Fiduccia-Mattheyses refinement under a balance tolerance: each side may
  // exceed its share by 2 % of that share
  const double tol = 0.02 * std::min(target, W - target) + 1e-12;
  double ws[2] = {0.0, 0.0};
  for (int u : nodes) ws[side[u]] += g.nw[u];
  for (int pass = 0; pass < 8; pass++) {
    std::map<int, double> gmap;
    auto gain_of = [&](int u) {
      double ext = 0.0, inn = 0.0;
      for (int e = g.ptr[u]; e < g.ptr[u + 1]; e++) {
        int v = g.adj[e];
        if (!in[v]) continue;
        (side[v] == side[u] ? inn : ext) += g.ew[e];
      }
      return ext - inn;
    };
    std::set<std::pair<double, int>> pq;  // (-gain, node): best gain first
    for (int u : nodes) {
      double gu = gain_of(u);
      gmap[u] = gu;
      pq.insert({-gu, u});
    }
    std::map<int, char> lock;
    std::vector<int> moved;
    double cum = 0.0, best = 0.0;
    size_t best_len = 0;
    while (!pq.empty()) {
      // the best-gain node whose move keeps the balance
      auto it = pq.begin();
      for (; it != pq.end(); ++it) {
        int u = it->second;
        int s = side[u];
        double w1 = ws[1 - s] + g.nw[u], t1 = (s == 0 ? W - target : target);
        if (w1 <= t1 + tol) break;
      }
      if (it == pq.end()) break;
      int u = it->second;
      double gu = -it->first;
      pq.erase(it);
      lock[u] = 1;
      int s = side[u];
      side[u] = 1 - s;
      ws[s] -= g.nw[u];
      ws[1 - s] += g.nw[u];
      moved.push_back(u);
      cum += gu;
      if (cum > best + 1e-12) {
        best = cum;
        best_len = moved.size();
      }
      for (int e = g.ptr[u]; e < g.ptr[u + 1]; e++) {
        int v = g.adj[e];
        if (!in[v] || lock.count(v)) continue;
        pq.erase({-gmap[v], v});
        gmap[v] = gain_of(v);
        pq.insert({-gmap[v], v});
      }
      if (moved.size() > best_len + 64) break;  // a long run without improvement
    }
    for (size_t a = moved.size(); a > best_len; a--) {  // back to the best prefix
      int u = moved[a - 1];
      int s = side[u];
      side[u] = 1 - s;
      ws[s] -= g.nw[u];
      ws[1 - s] += g.nw[u];
    }
    if (best_len == 0) break;
  }
}

void recurse(const Graph &g, std::vector<int> nodes, int k, int base, std::vector<char> &in, std::vector<int> &side,
             std::vector<int> &dist, int32_t *part) {
  if (k <= 1 || nodes.size() <= 1) {
    for (int u : nodes) part[u] = base;
    return;
  }
  int k0 = k / 2, k1 = k - k0;
  for (int u : nodes) in[u] = 1;
  bisect(g, nodes, in, (double)k0 / k, side, dist);
  for (int u : nodes) in[u] = 0;
  std::vector<int> a, b;
  for (int u : nodes) (side[u] == 0 ? a : b).push_back(u);
  if ((int)a.size() < k0 || (int)b.size() < k1) {
    // a side with fewer cameras than parts: share the nodes by weight order,
    // at least k0 to the first side and k1 to the second
    a.clear();
    b.clear();
    double W = 0.0, w = 0.0;
    for (int u : nodes) W += g.nw[u];
    const int n = (int)nodes.size();
    for (int u : nodes) {
      int na = (int)a.size();
      bool to_a = na < k0 || (w < W * k0 / k && n - na - 1 >= k1);
      (to_a ? a : b).push_back(u);
      w += g.nw[u];
    }
  }
  recurse(g, a, k0, base, in, side, dist, part);
  recurse(g, b, k1, base + k0, in, side, dist, part);
}

}  // namespace

extern "C" rpba_status rpba_partition(int32_t n_cams, int32_t n_points, int32_t n_obs, const int32_t *obs_cam,
                                      const int32_t *obs_point, int32_t n_parts, int32_t *cam_subblock,
                                      double *node_weight, double *edge_cut) {
  if (n_cams <= 0 || n_points < 0 || n_obs < 0 || n_parts < 1 || n_parts > n_cams || !cam_subblock ||
      (n_obs && (!obs_cam || !obs_point)))
    return RPBA_ERR_INVALID_ARG;
  for (int k = 0; k < n_obs; k++)
    if (obs_cam[k] < 0 || obs_cam[k] >= n_cams || obs_point[k] < 0 || obs_point[k] >= n_points)
      return RPBA_ERR_INVALID_ARG;
  Graph g;
  g.n = n_cams;
  // observations per point, and each point's cameras
  std::vector<int> cnt(n_points, 0);
  for (int k = 0; k < n_obs; k++) cnt[obs_point[k]]++;
  std::vector<int> pptr(n_points + 1, 0);
  for (int j = 0; j < n_points; j++) pptr[j + 1] = pptr[j] + cnt[j];
  std::vector<int> pcam(n_obs), fill(pptr.begin(), pptr.end() - 1);
  for (int k = 0; k < n_obs; k++) pcam[fill[obs_point[k]]++] = obs_cam[k];
  // node weights: cube root of the observation counts of the points seen
  std::vector<double> sum(n_cams, 0.0);
  for (int k = 0; k < n_obs; k++) sum[obs_cam[k]] += cnt[obs_point[k]];
  g.nw.resize(n_cams);
  for (int i = 0; i < n_cams; i++) g.nw[i] = cbrt(sum[i]);
  // edges: every pair of distinct cameras of a point, weighted by shared points
  std::vector<uint64_t> keys;
  for (int j = 0; j < n_points; j++) {
    std::vector<int> c(pcam.begin() + pptr[j], pcam.begin() + pptr[j + 1]);
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    for (size_t a = 0; a < c.size(); a++)
      for (size_t b = a + 1; b < c.size(); b++) {
        keys.push_back((uint64_t)c[a] << 32 | (uint32_t)c[b]);
        keys.push_back((uint64_t)c[b] << 32 | (uint32_t)c[a]);
      }
  }
  std::sort(keys.begin(), keys.end());
  g.ptr.assign(n_cams + 1, 0);
  for (size_t e = 0; e < keys.size();) {
    size_t f = e;
    while (f < keys.size() && keys[f] == keys[e]) f++;
    int a = (int)(keys[e] >> 32), b = (int)(keys[e] & 0xffffffffu);
    g.ptr[a + 1]++;
    g.adj.push_back(b);
    g.ew.push_back((double)(f - e));
    e = f;
  }
  for (int i = 0; i < n_cams; i++) g.ptr[i + 1] += g.ptr[i];
  std::vector<int> nodes(n_cams);
  std::iota(nodes.begin(), nodes.end(), 0);
  std::vector<char> in(n_cams, 0);
  std::vector<int> side(n_cams, 0), dist(n_cams, -1);
  recurse(g, nodes, n_parts, 0, in, side, dist, cam_subblock);
  if (node_weight)
    for (int i = 0; i < n_cams; i++) node_weight[i] = g.nw[i];
  if (edge_cut) {
    double c = 0.0;
    for (int u = 0; u < n_cams; u++)
      for (int e = g.ptr[u]; e < g.ptr[u + 1]; e++)
        if (g.adj[e] > u && cam_subblock[u] != cam_subblock[g.adj[e]]) c += g.ew[e];
    *edge_cut = c;
  }
  return RPBA_OK;
}
