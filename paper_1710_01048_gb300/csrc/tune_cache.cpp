// The batch autotuner's persisted cache (host only).
//
// The file is a JSON object written with one entry per line:
//   {
//     "<key>": {"config": [chunk, u_ctas, ctas, schedule], "ms": mean_ms},
//     ...
//   }
// The reader accepts exactly that shape (whitespace aside); a line it does
// not recognise is skipped on lookup and dropped when the file is rewritten.
// A store rewrites the whole file through a temporary file and a rename, so
// a reader never sees half an entry.
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

namespace wq {

namespace {

struct Entry {
  std::string key;
  int cfg[4];
  double ms;
};

// Parses one line of the cache; false if it is not an entry.
bool parse_line(const char *line, Entry *E) {
  const char *q0 = std::strchr(line, '"');
  if (!q0) return false;
  const char *q1 = std::strchr(q0 + 1, '"');
  if (!q1) return false;
  E->key.assign(q0 + 1, q1);
  const char *c = std::strstr(q1 + 1, "\"config\"");
  if (!c) return false;
  c = std::strchr(c, '[');
  if (!c) return false;
  c++;
  for (int i = 0; i < 4; i++) {
    char *end = nullptr;
    const long v = std::strtol(c, &end, 10);
    if (end == c || v < 0 || v > 1024) return false;
    E->cfg[i] = (int)v;
    c = end;
    while (*c == ' ' || *c == '\t') c++;
    if (i < 3) {
      if (*c != ',') return false;
      c++;
    } else if (*c != ']') {
      return false;
    }
  }
  const char *m = std::strstr(c, "\"ms\"");
  if (!m) return false;
  m = std::strchr(m + 4, ':');
  if (!m) return false;
  char *end = nullptr;
  E->ms = std::strtod(m + 1, &end);
  return end != m + 1;
}

std::vector<Entry> read_all(const char *path) {
  std::vector<Entry> out;
  FILE *f = std::fopen(path, "r");
  if (!f) return out;
  char buf[1024];
  while (std::fgets(buf, sizeof(buf), f)) {
    Entry E;
    if (parse_line(buf, &E)) out.push_back(E);
  }
  std::fclose(f);
  return out;
}

}  // namespace

// Keys carry no quote or backslash (they are written inside a JSON string).
std::string tune_cache_clean_key(const std::string &raw) {
  std::string k = raw;
  for (char &ch : k)
    if (ch == '"' || ch == '\\' || ch == '\n' || ch == '\r') ch = '_';
  return k;
}

bool tune_cache_lookup(const char *path, const std::string &key, int cfg[4], double *ms) {
  if (!path || !*path) return false;
  for (const Entry &E : read_all(path))
    if (E.key == key) {
      std::memcpy(cfg, E.cfg, sizeof(E.cfg));
      *ms = E.ms;
      return true;
    }
  return false;
}

bool tune_cache_store(const char *path, const std::string &key, const int cfg[4], double ms) {
  if (!path || !*path) return false;
  std::vector<Entry> all = read_all(path);
  bool found = false;
  for (Entry &E : all)
    if (E.key == key) {
      std::memcpy(E.cfg, cfg, sizeof(E.cfg));
      E.ms = ms;
      found = true;
    }
  if (!found) {
    Entry E;
    E.key = key;
    std::memcpy(E.cfg, cfg, sizeof(E.cfg));
    E.ms = ms;
    all.push_back(E);
  }
  const std::string tmp = std::string(path) + ".tmp." + std::to_string((long)getpid());
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  bool ok = std::fprintf(f, "{\n") > 0;
  for (size_t i = 0; i < all.size() && ok; i++)
    ok = std::fprintf(f, "  \"%s\": {\"config\": [%d, %d, %d, %d], \"ms\": %.6g}%s\n", all[i].key.c_str(),
                      all[i].cfg[0], all[i].cfg[1], all[i].cfg[2], all[i].cfg[3], all[i].ms,
                      i + 1 < all.size() ? "," : "") > 0;
  ok = ok && std::fprintf(f, "}\n") > 0;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return false;
  }
  return true;
}

}  // namespace wq
