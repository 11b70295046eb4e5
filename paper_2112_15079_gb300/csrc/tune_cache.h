// Persistent autotuner results: a small JSON file of tuned work
// decompositions, keyed by what decides the best one (precision,
// integrator, size class of the work, number of SMs) and by a hash of the
// kernel sources, so an entry taken on other kernels is never used.  Plain
// C++ without CUDA, so the library and a CPU test build the same code.
//
// File format (one object; entries in any order):
//   {"format": "nbody-tune-cache", "version": 1, "entries": [
//     {"precision": 1, "integrator": 0, "n_log2": 13, "systems_log2": 0,
//      "sms": 152, "kernels": "<hex>", "threads": 512, "ipt": 1, "tj": 1024,
//      "jsplit": 0, "ctas_per_sm": 2, "ms_per_step": 0.0674}, ...]}
// n_log2 / systems_log2 are floor(log2(bodies)) and floor(log2(systems)).
//
// Reading never fails loudly: a missing, unreadable or malformed file, an
// entry with missing or non-integer fields, or one whose key differs simply
// yields no entry (the caller keeps its defaults).  Writing replaces the
// entry with the same key, keeps the other well-formed entries, and goes
// through a temporary file renamed over the old one, so a reader never sees
// half a file; a malformed old file is replaced by one holding the new entry.
#pragma once

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <map>
#include <string>
#include <vector>

#include <unistd.h>

namespace nb {

struct TuneKey {
  int precision = 0, integrator = 0, n_log2 = 0, systems_log2 = 0, sms = 0;
  std::string kernels;
};

struct TuneEntry {
  int threads = 0, ipt = 0, tj = 0, jsplit = 0, ctas_per_sm = 0;
  double ms_per_step = 0.0;
};

inline int floor_log2(long long v) {
  int k = 0;
  while (v > 1) {
    v >>= 1;
    ++k;
  }
  return k;
}

// ---- a minimal JSON reader (objects, arrays, strings, numbers, literals) ----
struct JVal {
  enum Kind { kNull, kBool, kNum, kStr, kArr, kObj } kind = kNull;
  double num = 0.0;
  bool b = false;
  std::string str;
  std::vector<JVal> arr;
  std::map<std::string, JVal> obj;
};

class JParser {
 public:
  explicit JParser(const std::string &t) : t_(t) {}
  bool parse(JVal &out) {
    if (!value(out, 0)) return false;
    ws();
    return i_ == t_.size();
  }

 private:
  const std::string &t_;
  size_t i_ = 0;
  void ws() {
    while (i_ < t_.size() && (t_[i_] == ' ' || t_[i_] == '\n' || t_[i_] == '\r' || t_[i_] == '\t')) ++i_;
  }
  bool lit(const char *w) {
    size_t k = 0;
    while (w[k]) {
      if (i_ + k >= t_.size() || t_[i_ + k] != w[k]) return false;
      ++k;
    }
    i_ += k;
    return true;
  }
  bool string(std::string &s) {
    if (i_ >= t_.size() || t_[i_] != '"') return false;
    ++i_;
    s.clear();
    while (i_ < t_.size() && t_[i_] != '"') {
      char ch = t_[i_++];
      if (ch == '\\') {
        if (i_ >= t_.size()) return false;
        const char e = t_[i_++];
        if (e == 'n') ch = '\n';
        else if (e == 't') ch = '\t';
        else if (e == '"' || e == '\\' || e == '/') ch = e;
        else return false;  // (\u escapes are never written by this file's writer)
      }
      s.push_back(ch);
    }
    if (i_ >= t_.size()) return false;
    ++i_;
    return true;
  }
  bool value(JVal &v, int depth) {
    if (depth > 16) return false;
    ws();
    if (i_ >= t_.size()) return false;
    const char c = t_[i_];
    if (c == '{') {
      ++i_;
      v.kind = JVal::kObj;
      ws();
      if (i_ < t_.size() && t_[i_] == '}') {
        ++i_;
        return true;
      }
      for (;;) {
        ws();
        std::string k;
        if (!string(k)) return false;
        ws();
        if (i_ >= t_.size() || t_[i_] != ':') return false;
        ++i_;
        if (!value(v.obj[k], depth + 1)) return false;
        ws();
        if (i_ < t_.size() && t_[i_] == ',') {
          ++i_;
          continue;
        }
        if (i_ < t_.size() && t_[i_] == '}') {
          ++i_;
          return true;
        }
        return false;
      }
    }
    if (c == '[') {
      ++i_;
      v.kind = JVal::kArr;
      ws();
      if (i_ < t_.size() && t_[i_] == ']') {
        ++i_;
        return true;
      }
      for (;;) {
        v.arr.emplace_back();
        if (!value(v.arr.back(), depth + 1)) return false;
        ws();
        if (i_ < t_.size() && t_[i_] == ',') {
          ++i_;
          continue;
        }
        if (i_ < t_.size() && t_[i_] == ']') {
          ++i_;
          return true;
        }
        return false;
      }
    }
    if (c == '"') {
      v.kind = JVal::kStr;
      return string(v.str);
    }
    if (lit("true")) {
      v.kind = JVal::kBool;
      v.b = true;
      return true;
    }
    if (lit("false")) {
      v.kind = JVal::kBool;
      return true;
    }
    if (lit("null")) return true;
    const char *begin = t_.c_str() + i_;
    char *end = nullptr;
    const double d = std::strtod(begin, &end);
    if (end == begin || !std::isfinite(d)) return false;
    i_ += static_cast<size_t>(end - begin);
    v.kind = JVal::kNum;
    v.num = d;
    return true;
  }
};

inline bool read_file(const std::string &path, std::string &out) {
  std::FILE *f = std::fopen(path.c_str(), "rb");
  if (!f) return false;
  out.clear();
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) {
    out.append(buf, n);
    if (out.size() > (16u << 20)) {  // not a cache this library wrote
      std::fclose(f);
      return false;
    }
  }
  const bool ok = !std::ferror(f);
  std::fclose(f);
  return ok;
}

// An integer field of an entry (false if missing or not an integer).
inline bool jint(const JVal &o, const char *k, int &out) {
  auto it = o.obj.find(k);
  if (it == o.obj.end() || it->second.kind != JVal::kNum) return false;
  const double d = it->second.num;
  if (d != std::floor(d) || std::fabs(d) > 2147483647.0) return false;
  out = static_cast<int>(d);
  return true;
}

// One well-formed entry of a parsed file: its key and tiles.
inline bool tune_parse_entry(const JVal &e, TuneKey &k, TuneEntry &t) {
  if (e.kind != JVal::kObj) return false;
  auto ks = e.obj.find("kernels");
  if (ks == e.obj.end() || ks->second.kind != JVal::kStr) return false;
  k.kernels = ks->second.str;
  if (!jint(e, "precision", k.precision) || !jint(e, "integrator", k.integrator) || !jint(e, "n_log2", k.n_log2) ||
      !jint(e, "systems_log2", k.systems_log2) || !jint(e, "sms", k.sms))
    return false;
  if (!jint(e, "threads", t.threads) || !jint(e, "ipt", t.ipt) || !jint(e, "tj", t.tj) ||
      !jint(e, "jsplit", t.jsplit) || !jint(e, "ctas_per_sm", t.ctas_per_sm))
    return false;
  auto ms = e.obj.find("ms_per_step");
  t.ms_per_step = (ms != e.obj.end() && ms->second.kind == JVal::kNum) ? ms->second.num : 0.0;
  return true;
}

inline bool same_key(const TuneKey &a, const TuneKey &b) {
  return a.precision == b.precision && a.integrator == b.integrator && a.n_log2 == b.n_log2 &&
         a.systems_log2 == b.systems_log2 && a.sms == b.sms && a.kernels == b.kernels;
}

// All well-formed entries of the file at `path` (false if the file is
// missing or is not a cache of this format and version).
inline bool tune_read_all(const std::string &path, std::vector<std::pair<TuneKey, TuneEntry>> &out) {
  out.clear();
  std::string text;
  if (!read_file(path, text)) return false;
  JVal root;
  if (!JParser(text).parse(root) || root.kind != JVal::kObj) return false;
  auto fmt = root.obj.find("format");
  int version = 0;
  if (fmt == root.obj.end() || fmt->second.kind != JVal::kStr || fmt->second.str != "nbody-tune-cache" ||
      !jint(root, "version", version) || version != 1)
    return false;
  auto ent = root.obj.find("entries");
  if (ent == root.obj.end() || ent->second.kind != JVal::kArr) return false;
  for (const JVal &e : ent->second.arr) {
    TuneKey k;
    TuneEntry t;
    if (tune_parse_entry(e, k, t)) out.emplace_back(k, t);
  }
  return true;
}

// The entry for `key`, if the file holds a well-formed one.
inline bool tune_cache_lookup(const std::string &path, const TuneKey &key, TuneEntry &out) {
  std::vector<std::pair<TuneKey, TuneEntry>> all;
  if (!tune_read_all(path, all)) return false;
  for (const auto &kv : all)
    if (same_key(kv.first, key)) {
      out = kv.second;
      return true;
    }
  return false;
}

inline std::string json_escape(const std::string &s) {
  std::string o;
  for (char c : s) {
    if (c == '"' || c == '\\') o.push_back('\\');
    if (c == '\n') {
      o += "\\n";
      continue;
    }
    o.push_back(c);
  }
  return o;
}

// Add or replace the entry for `key`.  Returns "" on success, else why not.
inline std::string tune_cache_store(const std::string &path, const TuneKey &key, const TuneEntry &t) {
  std::vector<std::pair<TuneKey, TuneEntry>> all;
  tune_read_all(path, all);  // a missing or malformed file: start a new one
  bool replaced = false;
  for (auto &kv : all)
    if (same_key(kv.first, key)) {
      kv.second = t;
      replaced = true;
    }
  if (!replaced) all.emplace_back(key, t);
  std::string text = "{\"format\": \"nbody-tune-cache\", \"version\": 1, \"entries\": [";
  char buf[512];
  for (size_t i = 0; i < all.size(); ++i) {
    const TuneKey &k = all[i].first;
    const TuneEntry &e = all[i].second;
    std::snprintf(buf, sizeof buf,
                  "%s\n  {\"precision\": %d, \"integrator\": %d, \"n_log2\": %d, \"systems_log2\": %d, \"sms\": %d, "
                  "\"kernels\": \"%s\", \"threads\": %d, \"ipt\": %d, \"tj\": %d, \"jsplit\": %d, "
                  "\"ctas_per_sm\": %d, \"ms_per_step\": %.9g}",
                  i ? "," : "", k.precision, k.integrator, k.n_log2, k.systems_log2, k.sms,
                  json_escape(k.kernels).substr(0, 128).c_str(), e.threads, e.ipt, e.tj, e.jsplit, e.ctas_per_sm,
                  std::isfinite(e.ms_per_step) ? e.ms_per_step : 0.0);
    text += buf;
  }
  text += "\n]}\n";
  static std::atomic<unsigned> seq{0};
  const std::string tmp = path + ".tmp" + std::to_string(static_cast<long long>(getpid())) + "." +
                          std::to_string(seq.fetch_add(1));
  std::FILE *f = std::fopen(tmp.c_str(), "wb");
  if (!f) return "cannot create " + tmp;
  const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
  if (std::fclose(f) != 0 || !ok) {
    std::remove(tmp.c_str());
    return "cannot write " + tmp;
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return "cannot rename " + tmp + " to " + path;
  }
  return "";
}

}  // namespace nb
