// tune.cpp — the tuning registry: named integer knobs (kernel variant, tile
// rows, split factors) that the launchers read and the autotuner sets.  Unset
// knobs return the launcher's default.  Thread-safe; values are global to the
// process.
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "../../include/msketch.h"

namespace {
std::mutex g_mu;
std::map<std::string, long long>& table() {
  static std::map<std::string, long long> t;
  return t;
}
}  // namespace

namespace msk {
long long tune_get(const char* name, long long dflt) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = table().find(name);
  return it == table().end() ? dflt : it->second;
}
}  // namespace msk

extern "C" {

int msk_tune_set(const char* name, long long value) {
  if (!name || !*name) return -1;
  std::lock_guard<std::mutex> lock(g_mu);
  table()[name] = value;
  return MSK_OK;
}

int msk_tune_clear(const char* name) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!name) {
    table().clear();
  } else {
    table().erase(name);
  }
  return MSK_OK;
}

long long msk_tune_get(const char* name, long long dflt) { return msk::tune_get(name, dflt); }

}  // extern "C"
