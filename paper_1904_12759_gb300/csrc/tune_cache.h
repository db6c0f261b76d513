// Schedule cache of the batch autotuners (host code): a small text file with
// one JSON object per line, {"key": "<signature>", "<field>": <integer>, ...,
// "ms": <tuned time>}; the last line with a matching key wins.
#pragma once

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <utility>
#include <vector>

namespace mcx {

// Integer `field` of the last line whose key equals `key`; false if none.
inline bool tune_cache_get(const char *path, const std::string &key, const char *field, long *out) {
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    const std::string needle = "\"key\": \"" + key + "\"";
    const std::string fname = std::string("\"") + field + "\": ";
    while (fgets(line, sizeof line, f)) {
        if (!strstr(line, needle.c_str())) continue;
        const char *c = strstr(line, fname.c_str());
        if (c) {
            *out = strtol(c + fname.size(), nullptr, 10);
            found = true;
        }
    }
    fclose(f);
    return found;
}

inline void tune_cache_put(const char *path, const std::string &key,
                           const std::vector<std::pair<const char *, long>> &fields, double ms) {
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\"", key.c_str());
    for (const auto &kv : fields) fprintf(f, ", \"%s\": %ld", kv.first, kv.second);
    fprintf(f, ", \"ms\": %.4f}\n", ms);
    fclose(f);
}

}  // namespace mcx
