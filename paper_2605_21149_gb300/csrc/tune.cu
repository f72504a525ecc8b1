// Tuning table: named integer settings plus the tile shapes the float64 GEMM
// autotuner has measured, one process-wide table behind a mutex.
//
// Keys in use:
//   dgemm_autotune   1 (default): time every tile candidate the first time a
//                    small or medium float64 product shape is met (C at most
//                    2^24 entries, K at most 4096, C not aliasing A or B, the
//                    stream not capturing) and keep the fastest; 0: built-in
//                    heuristic only
//   dgemm:<ta>,<tb>,<lower>,<M>,<N>,<K>,<alias>   measured tile, 10 RM + RN
//   batch_streams    worker streams of pix_loglike_batch (default 4, 1..16)
//   ozaki_stages     3 (default) / 2: depth of the split kernel's TMA ring
//   emu_tc           1 (default) / 0: emulator inference layers on tcgen05
//                    / all through the WMMA product
//   emu_tc0          1 (default) / 0: with emu_tc, the first layer too (its
//                    16 inputs widened with zeros to 64) / on WMMA
//   split_diag_df    0 (default): the split-precision Cholesky factors its
//                    64-wide diagonal blocks and their row solves in float64;
//                    1: in float-float (pairs of float32, about 2^-46 per
//                    operation; faster on this part's narrow float64 pipe)
//   batch_split_kt   0 (default): with split-precision masks the per-item
//                    inner factor Kt of pix_loglike_batch is native float64;
//                    1: its trailing updates and panel products are split
//   test_wait_timeout  1: failure-path test; the split-precision kernel
//                    issues no copies and gives up each wait after 1 ms
//   batch_graphs     1 (default): pix_loglike_batch captures each worker's
//                    per-item sequence once per mask as a CUDA graph and
//                    replays it; 0: plain launches
// The text form is one "key value" pair per line.
#include "qmlgb.h"
#include "internal.cuh"

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

namespace qmlgb {

namespace {
std::mutex g_tune_mu;
std::map<std::string, int64_t> &table() {
  static std::map<std::string, int64_t> t;
  return t;
}
}  // namespace

int64_t tune_get(const std::string &key, int64_t dflt) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = table().find(key);
  return it == table().end() ? dflt : it->second;
}

bool tune_find(const std::string &key, int64_t &value) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = table().find(key);
  if (it == table().end()) return false;
  value = it->second;
  return true;
}

void tune_put(const std::string &key, int64_t value) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  table()[key] = value;
}

void set_last_error(const std::string &msg);

}  // namespace qmlgb

using namespace qmlgb;

namespace {
bool valid_key(const char *key) {
  if (!key || !*key) return false;
  for (const char *p = key; *p; ++p)
    if (*p == ' ' || *p == '\n' || *p == '\t' || *p == '\r') return false;
  return true;
}
}  // namespace

extern "C" {

qml_status qml_tune_set(const char *key, int64_t value) {
  if (!valid_key(key)) {
    set_last_error("qml_tune_set: key must be non-empty without white space");
    return QML_EINVAL;
  }
  tune_put(key, value);
  return QML_OK;
}

qml_status qml_tune_get(const char *key, int64_t *value) {
  if (!valid_key(key) || !value) {
    set_last_error("qml_tune_get: bad arguments");
    return QML_EINVAL;
  }
  if (!tune_find(key, *value)) {
    set_last_error(std::string("qml_tune_get: no entry ") + key);
    return QML_EINVAL;
  }
  return QML_OK;
}

int64_t qml_tune_table(char *buf, int64_t cap) {
  std::string s;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (const auto &kv : table()) s += kv.first + " " + std::to_string(kv.second) + "\n";
  }
  const int64_t need = (int64_t)s.size() + 1;
  if (buf && cap >= need) memcpy(buf, s.c_str(), (size_t)need);
  return need;
}

qml_status qml_tune_load(const char *text) {
  if (!text) {
    set_last_error("qml_tune_load: NULL text");
    return QML_EINVAL;
  }
  std::istringstream in(text);
  std::string line;
  int lineno = 0;
  std::map<std::string, int64_t> parsed;
  while (std::getline(in, line)) {
    ++lineno;
    if (line.empty() || line[0] == '#') continue;
    std::istringstream ls(line);
    std::string key;
    long long v;
    std::string rest;
    if (!(ls >> key >> v) || (ls >> rest)) {
      set_last_error("qml_tune_load: line " + std::to_string(lineno) + " is not 'key value'");
      return QML_EINVAL;
    }
    parsed[key] = (int64_t)v;
  }
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (const auto &kv : parsed) table()[kv.first] = kv.second;
  return QML_OK;
}

}  // extern "C"
