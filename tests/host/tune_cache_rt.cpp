// Host harness of the autotuner's JSON cache (tune_cache.h): "write PATH K V [K V ...]" writes the
// pairs; "read PATH" prints "ok" and one "KEY<TAB>VALUE" line per entry, or "bad".
#include <cstdio>
#include <cstring>
#include <map>
#include <string>

#include "tune_cache.h"

int main(int argc, char** argv) {
  if (argc >= 3 && std::strcmp(argv[1], "write") == 0) {
    std::map<std::string, std::string> m;
    for (int i = 3; i + 1 < argc; i += 2) m[argv[i]] = argv[i + 1];
    return sl::write_tune_cache(argv[2], m) ? 0 : 1;
  }
  if (argc == 3 && std::strcmp(argv[1], "read") == 0) {
    std::map<std::string, std::string> m;
    if (!sl::read_tune_cache(argv[2], m)) {
      std::puts("bad");
      return 0;
    }
    std::puts("ok");
    for (const auto& kv : m) std::printf("%s\t%s\n", kv.first.c_str(), kv.second.c_str());
    return 0;
  }
  return 2;
}
