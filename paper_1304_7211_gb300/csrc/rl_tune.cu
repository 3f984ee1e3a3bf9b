// rl_tune.cu -- the autotuner's choice cache (host code).
//
// A tuned choice is keyed by the request alone -- tunable site, its PSF
// parameter, image size, storage, boundary, thinning and the device's SM
// count -- never by what else runs, so a request keeps its choice in any
// mix.  The cache is process-wide; with RL_TUNE_CACHE set to a file name it
// is read from that file on first use and every new choice is appended to it
// as one JSON object per line:
//   {"key": "disc-launch:r12:4096x4096:f32:mirror:plain:sm152", "choice": 6, "us": "137.4 133.5 126.6"}
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "rl_launch.h"

namespace rl {
namespace {

std::mutex g_mu;
std::map<std::string, int> g_cache;
bool g_loaded = false;

const char *cache_file() {
    const char *p = std::getenv("RL_TUNE_CACHE");
    return p && *p ? p : nullptr;
}

// One entry per line; lines that do not parse are skipped.
void load_locked() {
    g_loaded = true;
    const char *path = cache_file();
    if (!path) return;
    FILE *fh = std::fopen(path, "r");
    if (!fh) return;
    char line[1024];
    while (std::fgets(line, sizeof line, fh)) {
        char key[512];
        int choice = 0;
        const char *k = std::strstr(line, "\"key\": \"");
        const char *c = std::strstr(line, "\"choice\": ");
        if (!k || !c) continue;
        if (std::sscanf(k + 8, "%511[^\"]", key) == 1 && std::sscanf(c + 10, "%d", &choice) == 1)
            g_cache[key] = choice;
    }
    std::fclose(fh);
}

}  // namespace

bool tune_get(const std::string &key, int *choice) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_loaded) load_locked();
    auto it = g_cache.find(key);
    if (it == g_cache.end()) return false;
    *choice = it->second;
    return true;
}

void tune_put(const std::string &key, int choice, const std::string &timings_us) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_loaded) load_locked();
    g_cache[key] = choice;
    const char *path = cache_file();
    if (!path) return;
    if (FILE *fh = std::fopen(path, "a")) {
        std::fprintf(fh, "{\"key\": \"%s\", \"choice\": %d, \"us\": \"%s\"}\n", key.c_str(), choice,
                     timings_us.c_str());
        std::fclose(fh);
    }
}

void tune_clear() {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache.clear();
    g_loaded = false;
}

}  // namespace rl
