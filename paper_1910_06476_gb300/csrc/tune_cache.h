#pragma once
// JSON cache of the launch-shape autotuner (sl_tune): one flat JSON object of string keys and
// string values.  Keys and values are built by the library from names, numbers and separators,
// so no escapes are read or written; anything else is rejected.  Host code only.
#include <cstdio>
#include <map>
#include <string>

namespace sl {

inline bool read_tune_cache(const std::string& path, std::map<std::string, std::string>& out) {
  out.clear();
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return true;                       // no file yet: an empty cache
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
  std::fclose(f);
  size_t i = 0;
  auto skip = [&] {
    while (i < text.size() && (text[i] == ' ' || text[i] == '\n' || text[i] == '\r' || text[i] == '\t')) ++i;
  };
  auto str = [&](std::string& s) {
    skip();
    if (i >= text.size() || text[i] != '"') return false;
    const size_t e = text.find('"', i + 1);
    if (e == std::string::npos) return false;
    s = text.substr(i + 1, e - i - 1);
    i = e + 1;
    return true;
  };
  skip();
  if (i >= text.size()) return true;
  if (text[i] != '{') return false;
  ++i;
  skip();
  if (i < text.size() && text[i] == '}') return true;
  for (;;) {
    std::string key, val;
    if (!str(key)) return false;
    skip();
    if (i >= text.size() || text[i] != ':') return false;
    ++i;
    if (!str(val)) return false;
    out[key] = val;
    skip();
    if (i < text.size() && text[i] == ',') { ++i; continue; }
    if (i < text.size() && text[i] == '}') return true;
    return false;
  }
}

inline bool write_tune_cache(const std::string& path, const std::map<std::string, std::string>& m) {
  const std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  std::fputs("{\n", f);
  size_t k = 0;
  for (const auto& kv : m)
    std::fprintf(f, "  \"%s\": \"%s\"%s\n", kv.first.c_str(), kv.second.c_str(), ++k < m.size() ? "," : "");
  std::fputs("}\n", f);
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), path.c_str()) == 0;
}

}  // namespace sl
