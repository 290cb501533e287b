// Process-wide table of harvest launch settings chosen by the autotuner,
// keyed by what decides the harvest kernel's shape, its visited sets and the
// length of its neighbour lists: the metric, the dimension, the beam width,
// the degree bound, ceil(log2 n), the number of trees and of blocks.
// Saved and loaded as JSON of one fixed form:
//   {"fgraft_tuning": 1, "entries": [
//     {"metric": 1, "d": 100, "ef_h": 100, "R": 64, "log2_n": 21, "T": 8, "B": 8,
//      "warps_per_cta": 4, "hash_log2": 0, "overflow_mode": 1, "gather": 1,
//      "id_batch": 2, "us_per_query": 0.95}, ...]}
// ("gather" and "id_batch" may be absent: 0 and 2).
// hash_log2 0 keeps the occupancy rule for the visited-set layout.
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "internal.h"

namespace fg {

namespace {

using Key = std::tuple<int, int, int, int, int, int, int>;

std::mutex& table_mu() {
  static std::mutex mu;
  return mu;
}
std::map<Key, TuneVal>& table() {
  static std::map<Key, TuneVal> t;
  return t;
}

Key key_of(const TuneKey& k) { return Key{k.metric, k.d, k.ef, k.R, k.log2_n, k.T, k.B}; }

// Value of "name": <number> inside [b, e), or false.
bool field(const char* b, const char* e, const char* name, double* out) {
  const std::string pat = std::string("\"") + name + "\"";
  const char* p = b;
  while (p < e) {
    const char* q = strstr(p, pat.c_str());
    if (!q || q >= e) return false;
    q += pat.size();
    while (q < e && (*q == ' ' || *q == '\t' || *q == '\n' || *q == '\r')) ++q;
    if (q < e && *q == ':') {
      ++q;
      char* end = nullptr;
      errno = 0;
      const double v = strtod(q, &end);
      if (end == q || end > e || errno) return false;
      *out = v;
      return true;
    }
    p = q;
  }
  return false;
}

}  // namespace

bool tune_table_lookup(const TuneKey& k, TuneVal* v) {
  std::lock_guard<std::mutex> lock(table_mu());
  auto it = table().find(key_of(k));
  if (it == table().end()) return false;
  *v = it->second;
  return true;
}

void tune_table_put(const TuneKey& k, const TuneVal& v) {
  std::lock_guard<std::mutex> lock(table_mu());
  table()[key_of(k)] = v;
}

int tune_table_size() {
  std::lock_guard<std::mutex> lock(table_mu());
  return (int)table().size();
}

int tune_table_save(const char* path) {
  std::lock_guard<std::mutex> lock(table_mu());
  FILE* f = fopen(path, "w");
  if (!f) {
    set_error(1, std::string("cannot write ") + path);
    return 1;
  }
  fprintf(f, "{\"fgraft_tuning\": 1, \"entries\": [");
  bool first = true;
  for (const auto& kv : table()) {
    const Key& k = kv.first;
    const TuneVal& v = kv.second;
    fprintf(f,
            "%s\n  {\"metric\": %d, \"d\": %d, \"ef_h\": %d, \"R\": %d, \"log2_n\": %d, "
            "\"T\": %d, \"B\": %d, \"warps_per_cta\": %d, \"hash_log2\": %d, "
            "\"overflow_mode\": %d, \"gather\": %d, \"id_batch\": %d, \"us_per_query\": %.6g}",
            first ? "" : ",", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
            std::get<4>(k), std::get<5>(k), std::get<6>(k), v.wpc, v.hash_log2, v.overflow,
            v.gather, v.id_batch, v.us_per_query);
    first = false;
  }
  fprintf(f, "\n]}\n");
  const bool bad = ferror(f) != 0;
  fclose(f);
  if (bad) {
    set_error(1, std::string("error writing ") + path);
    return 1;
  }
  return 0;
}

int tune_table_load(const char* path) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_error(1, std::string("cannot read ") + path);
    return 1;
  }
  std::string txt;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, got);
  fclose(f);
  const char* s = txt.c_str();
  const char* ent = strstr(s, "\"entries\"");
  if (!strstr(s, "\"fgraft_tuning\"") || !ent) {
    set_error(1, std::string(path) + " is not an fgraft tuning table");
    return 1;
  }
  std::map<Key, TuneVal> loaded;
  const char* p = strchr(ent, '[');
  while (p) {
    const char* b = strchr(p, '{');
    if (!b) break;
    const char* e = strchr(b, '}');
    if (!e) {
      set_error(1, std::string(path) + ": unterminated entry");
      return 1;
    }
    double m, d, ef, R, ln, T, B, w, h, o, us = 0.0;
    if (!field(b, e, "metric", &m) || !field(b, e, "d", &d) || !field(b, e, "ef_h", &ef) ||
        !field(b, e, "R", &R) || !field(b, e, "log2_n", &ln) || !field(b, e, "T", &T) ||
        !field(b, e, "B", &B) ||
        !field(b, e, "warps_per_cta", &w) || !field(b, e, "hash_log2", &h) ||
        !field(b, e, "overflow_mode", &o)) {
      set_error(1, std::string(path) + ": entry without a required field");
      return 1;
    }
    field(b, e, "us_per_query", &us);
    double ga = 0.0, ib = 2.0;
    field(b, e, "gather", &ga);
    field(b, e, "id_batch", &ib);
    if (w < 1 || w > 4 || (h != 0 && (h < 7 || h > 14)) || o < 1 || o > 2 || ga < 0 ||
        ga > 1 || ib < 1 || ib > 2) {
      set_error(1, std::string(path) + ": entry with a setting out of range");
      return 1;
    }
    TuneVal v{(int)w, (int)h, (int)o, (int)ga, (int)ib, (float)us};
    loaded[Key{(int)m, (int)d, (int)ef, (int)R, (int)ln, (int)T, (int)B}] = v;
    p = e + 1;
  }
  std::lock_guard<std::mutex> lock(table_mu());
  for (const auto& kv : loaded) table()[kv.first] = kv.second;
  return 0;
}

}  // namespace fg
