// Admission core of the request loop (include/q2_serve.h): FIFO queue, byte
// ledger against a device-memory budget (running workspaces plus the resident
// tables of every problem the loop keeps), LRU eviction of unused problems,
// slot limit, queue timeout and latency statistics.  Host only.
#include <algorithm>
#include <cmath>
#include <deque>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/q2_serve.h"

struct q2_server {
  struct Entry {
    int64_t id;
    size_t bytes;
    int64_t problem;
    double t_submit;
  };
  struct Problem {
    size_t table_bytes = 0;
    int refs = 0;            // queued + running requests of this problem
    bool resident = false;   // its tables are charged to the ledger
    double last_use = 0;
  };
  size_t budget = 0;
  int max_slots = 0;
  double timeout = 0;
  std::deque<Entry> queue;
  std::unordered_map<int64_t, Entry> running;
  std::unordered_map<int64_t, int> seen;
  std::unordered_map<int64_t, Problem> problems;
  std::vector<int64_t> evicted;   // problems whose tables the caller should release
  size_t work_bytes = 0, table_bytes = 0, high_water = 0;
  int64_t submitted = 0, admitted = 0, completed = 0, expired = 0, evictions = 0;
  std::vector<double> latencies;
  mutable std::mutex mu;

  size_t in_use() const { return work_bytes + table_bytes; }

  // Release resident tables of unused problems, least recently used first,
  // until `need` more bytes fit the budget.  Returns whether they fit.
  bool make_room(size_t need, int64_t keep) {
    while (in_use() + need > budget) {
      int64_t victim = 0;
      bool found = false;
      double oldest = 0;
      for (const auto &kv : problems) {
        const Problem &p = kv.second;
        if (!p.resident || p.refs > 0 || kv.first == keep) continue;
        if (!found || p.last_use < oldest || (p.last_use == oldest && kv.first < victim)) {
          victim = kv.first;
          oldest = p.last_use;
          found = true;
        }
      }
      if (!found) return false;
      Problem &p = problems[victim];
      table_bytes -= p.table_bytes;
      p.resident = false;
      evicted.push_back(victim);
      ++evictions;
      if (p.refs == 0) problems.erase(victim);
    }
    return true;
  }
};

extern "C" {

q2_status q2_server_create(size_t budget_bytes, int max_slots, double queue_timeout_s, q2_server **out) {
  if (!out || budget_bytes == 0 || max_slots < 1 || !(queue_timeout_s > 0)) return Q2_ERR_INVALID;
  q2_server *s = new (std::nothrow) q2_server;
  if (!s) return Q2_ERR_OOM;
  s->budget = budget_bytes;
  s->max_slots = max_slots;
  s->timeout = queue_timeout_s;
  *out = s;
  return Q2_OK;
}

q2_status q2_server_destroy(q2_server *server) {
  delete server;
  return Q2_OK;
}

q2_status q2_server_submit(q2_server *s, int64_t id, size_t bytes, int64_t problem, size_t table_bytes,
                           double now_s) {
  if (!s || now_s < 0) return Q2_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->seen.count(id)) return Q2_ERR_INVALID;
  auto it = s->problems.find(problem);
  const size_t tb = it != s->problems.end() && it->second.resident ? 0 : table_bytes;
  if (bytes + tb > s->budget || bytes + table_bytes > s->budget) return Q2_ERR_OOM;
  s->seen[id] = 1;
  q2_server::Problem &p = s->problems[problem];
  if (!p.resident) p.table_bytes = table_bytes;
  ++p.refs;
  p.last_use = std::max(p.last_use, now_s);
  s->queue.push_back({id, bytes, problem, now_s});
  ++s->submitted;
  return Q2_OK;
}

int q2_server_admit(q2_server *s, double now_s, int64_t *ids_out, int cap) {
  if (!s || (cap > 0 && !ids_out) || now_s < 0) return -1;
  std::lock_guard<std::mutex> g(s->mu);
  int k = 0;
  for (auto it = s->queue.begin(); it != s->queue.end() && k < cap;) {
    if ((int)s->running.size() >= s->max_slots) break;
    q2_server::Problem &p = s->problems[it->problem];
    const size_t need = it->bytes + (p.resident ? 0 : p.table_bytes);
    if (s->make_room(need, it->problem)) {
      if (!p.resident) {
        p.resident = true;
        s->table_bytes += p.table_bytes;
      }
      p.last_use = std::max(p.last_use, now_s);
      s->work_bytes += it->bytes;
      s->high_water = std::max(s->high_water, s->in_use());
      s->running[it->id] = *it;
      ids_out[k++] = it->id;
      ++s->admitted;
      it = s->queue.erase(it);
    } else {
      ++it;
    }
  }
  return k;
}

static void drop_ref(q2_server *s, int64_t problem, double now_s) {
  auto it = s->problems.find(problem);
  if (it == s->problems.end()) return;
  --it->second.refs;
  it->second.last_use = std::max(it->second.last_use, now_s);
  if (it->second.refs <= 0 && !it->second.resident) s->problems.erase(it);
}

int q2_server_expire(q2_server *s, double now_s, int64_t *ids_out, int cap) {
  if (!s || (cap > 0 && !ids_out) || now_s < 0) return -1;
  std::lock_guard<std::mutex> g(s->mu);
  int k = 0;
  for (auto it = s->queue.begin(); it != s->queue.end() && k < cap;) {
    if (now_s - it->t_submit > s->timeout) {
      ids_out[k++] = it->id;
      ++s->expired;
      drop_ref(s, it->problem, now_s);
      it = s->queue.erase(it);
    } else {
      ++it;
    }
  }
  return k;
}

q2_status q2_server_complete(q2_server *s, int64_t id, double now_s) {
  if (!s || now_s < 0) return Q2_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->running.find(id);
  if (it == s->running.end()) return Q2_ERR_INVALID;
  s->work_bytes -= it->second.bytes;
  s->latencies.push_back(now_s - it->second.t_submit);
  drop_ref(s, it->second.problem, now_s);
  s->running.erase(it);
  ++s->completed;
  return Q2_OK;
}

int q2_server_take_evicted(q2_server *s, int64_t *problems_out, int cap) {
  if (!s || (cap > 0 && !problems_out)) return -1;
  std::lock_guard<std::mutex> g(s->mu);
  const int k = (int)std::min<size_t>((size_t)std::max(cap, 0), s->evicted.size());
  for (int i = 0; i < k; ++i) problems_out[i] = s->evicted[i];
  s->evicted.erase(s->evicted.begin(), s->evicted.begin() + k);
  return k;
}

q2_status q2_server_stats(const q2_server *s, double *out) {
  if (!s || !out) return Q2_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  std::vector<double> lat = s->latencies;
  double p50 = 0, p99 = 0, mean = 0;
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto q = [&](double f) {
      const size_t i = (size_t)std::min<double>((double)lat.size() - 1, std::ceil(f * (double)lat.size()) - 1);
      return lat[i];
    };
    p50 = q(0.50);
    p99 = q(0.99);
    for (double v : lat) mean += v;
    mean /= (double)lat.size();
  }
  int64_t resident = 0;
  for (const auto &kv : s->problems) resident += kv.second.resident ? 1 : 0;
  out[0] = (double)s->submitted;
  out[1] = (double)s->admitted;
  out[2] = (double)s->completed;
  out[3] = (double)s->expired;
  out[4] = (double)s->queue.size();
  out[5] = (double)s->running.size();
  out[6] = (double)s->in_use();
  out[7] = (double)s->high_water;
  out[8] = p50;
  out[9] = p99;
  out[10] = mean;
  out[11] = (double)s->table_bytes;
  out[12] = (double)resident;
  out[13] = (double)s->evictions;
  return Q2_OK;
}

}  // extern "C"
