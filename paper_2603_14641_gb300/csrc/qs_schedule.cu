// Window scheduling on the host, Sec. 4.2 ("Parallel Gate and Measurement
// Scheduling on CPU", ScheduleWindows of Alg. 2).
//
// An ordered list of gates and Z-measurements is cut into windows: a window is
// either a maximal set of gates on pairwise disjoint qubits, every one of which
// is the first remaining operation on all of its qubits (gates advance as early
// as their dependencies allow), or one measurement. Measurements are barriers:
// after each window of gates, every measurement that has become the first
// remaining operation on its qubit is emitted, in ascending qubit order, each
// as a window of its own (or all of them as one window in sampling mode, the
// paper's remark on sampling). This ordering reproduces the paper's worked
// example (its circuit figure: W0 = {H q0, P q2, P q4}, W1 = M q1, W2 = M q3,
// W3 = {P q0, H q1, P q3}, W4 = {CX 0->2, CX 3->4}, W5 = {H q2, P q3}).
// Runs in O(operations + qubits log qubits) with a queue per qubit.
#include <algorithm>
#include <cstdio>
#include <queue>
#include <string>
#include <vector>

#include "qs_internal.cuh"

namespace {
thread_local std::string g_sched_err;
int sfail(int code, const char *msg) {
  g_sched_err = msg;
  return code;
}
bool two_q(uint32_t t) { return t >= QS_CX && t <= QS_ISWAP; }
}  // namespace

extern "C" {

const char *qs_schedule_last_error(void) { return g_sched_err.c_str(); }

int qs_schedule_windows(uint32_t n, const qs_gate *ops, uint32_t count, int merge_measurements,
                        qs_gate *out_ops, uint32_t *out_window_ptr, uint8_t *out_window_kind,
                        uint32_t *n_windows) {
  if (!n_windows || (count && (!ops || !out_ops || !out_window_ptr || !out_window_kind)))
    return sfail(QS_ERR_ARG, "NULL argument");
  if (n == 0) return sfail(QS_ERR_ARG, "n must be positive");
  // per-qubit queues of operation indices, in input order
  std::vector<uint32_t> qcount(n, 0);
  for (uint32_t i = 0; i < count; ++i) {
    const uint32_t t = ops[i].type;
    if (t > QS_MEASURE) return sfail(QS_ERR_ARG, "unknown operation type");
    if (ops[i].q0 >= n || (two_q(t) && (ops[i].q1 >= n || ops[i].q1 == ops[i].q0)))
      return sfail(QS_ERR_ARG, "qubit out of range or two-qubit gate on one qubit");
    qcount[ops[i].q0]++;
    if (two_q(t)) qcount[ops[i].q1]++;
  }
  std::vector<uint32_t> qstart(n + 1, 0);
  for (uint32_t q = 0; q < n; ++q) qstart[q + 1] = qstart[q] + qcount[q];
  std::vector<uint32_t> qlist(qstart[n]), head(n, 0), fill(n, 0);
  for (uint32_t i = 0; i < count; ++i) {
    const uint32_t a = ops[i].q0;
    qlist[qstart[a] + fill[a]++] = i;
    if (two_q(ops[i].type)) {
      const uint32_t b = ops[i].q1;
      qlist[qstart[b] + fill[b]++] = i;
    }
  }
  auto front = [&](uint32_t q) -> int64_t {
    return head[q] < qcount[q] ? (int64_t)qlist[qstart[q] + head[q]] : -1;
  };
  std::vector<uint8_t> queued(count, 0);
  std::vector<uint32_t> ready;  // gates ready for the next window
  std::priority_queue<uint32_t, std::vector<uint32_t>, std::greater<uint32_t>> meas;  // qubits
  auto consider = [&](uint32_t q) {
    const int64_t f = front(q);
    if (f < 0 || queued[f]) return;
    const qs_gate &g = ops[f];
    if (g.type == QS_MEASURE) {
      queued[f] = 1;
      meas.push(q);
      return;
    }
    if (two_q(g.type)) {
      if (front(g.q0) != f || front(g.q1) != f) return;
    }
    queued[f] = 1;
    ready.push_back((uint32_t)f);
  };
  for (uint32_t q = 0; q < n; ++q) consider(q);
  uint32_t out = 0, w = 0;
  out_window_ptr[0] = 0;
  std::vector<uint32_t> window, touched;
  while (out < count) {
    // 1. window of every ready gate (ascending input position)
    if (!ready.empty()) {
      window.swap(ready);
      ready.clear();
      std::sort(window.begin(), window.end());
      touched.clear();
      for (uint32_t f : window) {
        out_ops[out++] = ops[f];
        head[ops[f].q0]++;
        touched.push_back(ops[f].q0);
        if (two_q(ops[f].type)) {
          head[ops[f].q1]++;
          touched.push_back(ops[f].q1);
        }
      }
      out_window_kind[w] = 0;
      out_window_ptr[++w] = out;
      for (uint32_t q : touched) consider(q);
    }
    // 2. measurements now first on their qubits, ascending qubit order
    bool any = false;
    while (!meas.empty()) {
      const uint32_t q = meas.top();
      meas.pop();
      const int64_t f = front(q);
      out_ops[out++] = ops[f];
      head[q]++;
      any = true;
      if (!merge_measurements) {
        out_window_kind[w] = 1;
        out_window_ptr[++w] = out;
      }
      consider(q);
    }
    if (any && merge_measurements) {
      out_window_kind[w] = 1;
      out_window_ptr[++w] = out;
    }
    if (ready.empty() && meas.empty() && out < count)
      return sfail(QS_ERR_INTERNAL, "scheduler stalled");
  }
  *n_windows = w;
  return QS_OK;
}

}  // extern "C"
