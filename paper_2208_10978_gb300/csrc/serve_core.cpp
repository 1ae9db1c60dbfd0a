// Admission core of the request loop (include/q2_serve.h): FIFO queue,
// byte ledger against a device-memory budget, slot limit, queue timeout and
// latency statistics.  Host only.
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
    double t_submit;
  };
  size_t budget = 0;
  int max_slots = 0;
  double timeout = 0;
  std::deque<Entry> queue;
  std::unordered_map<int64_t, Entry> running;
  std::unordered_map<int64_t, int> seen;
  size_t in_use = 0, high_water = 0;
  int64_t submitted = 0, admitted = 0, completed = 0, expired = 0;
  std::vector<double> latencies;
  mutable std::mutex mu;
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

q2_status q2_server_submit(q2_server *s, int64_t id, size_t bytes, double now_s) {
  if (!s || now_s < 0) return Q2_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->seen.count(id)) return Q2_ERR_INVALID;
  if (bytes > s->budget) return Q2_ERR_OOM;
  s->seen[id] = 1;
  s->queue.push_back({id, bytes, now_s});
  ++s->submitted;
  return Q2_OK;
}

int q2_server_admit(q2_server *s, double now_s, int64_t *ids_out, int cap) {
  if (!s || (cap > 0 && !ids_out) || now_s < 0) return -1;
  std::lock_guard<std::mutex> g(s->mu);
  int k = 0;
  for (auto it = s->queue.begin(); it != s->queue.end() && k < cap;) {
    if ((int)s->running.size() >= s->max_slots) break;
    if (s->in_use + it->bytes <= s->budget) {
      s->in_use += it->bytes;
      s->high_water = std::max(s->high_water, s->in_use);
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

int q2_server_expire(q2_server *s, double now_s, int64_t *ids_out, int cap) {
  if (!s || (cap > 0 && !ids_out) || now_s < 0) return -1;
  std::lock_guard<std::mutex> g(s->mu);
  int k = 0;
  for (auto it = s->queue.begin(); it != s->queue.end() && k < cap;) {
    if (now_s - it->t_submit > s->timeout) {
      ids_out[k++] = it->id;
      ++s->expired;
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
  s->in_use -= it->second.bytes;
  s->latencies.push_back(now_s - it->second.t_submit);
  s->running.erase(it);
  ++s->completed;
  return Q2_OK;
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
  out[0] = (double)s->submitted;
  out[1] = (double)s->admitted;
  out[2] = (double)s->completed;
  out[3] = (double)s->expired;
  out[4] = (double)s->queue.size();
  out[5] = (double)s->running.size();
  out[6] = (double)s->in_use;
  out[7] = (double)s->high_water;
  out[8] = p50;
  out[9] = p99;
  out[10] = mean;
  return Q2_OK;
}

}  // extern "C"
