// Autotune table loading: a small JSON object written by the autotuner
// (paper_1008_3171_gb300/autotune.py), e.g. {"run": 32, "streams": 1, "grab": 8,
// "cta": 256, "limb_bump": 0, "wide_min_bits": 32}.  Unknown keys are ignored;
// missing or out-of-range values keep the built-in defaults.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "bbp_runtime.h"

namespace bbp {

namespace {
bool read_int(const std::string& text, const char* key, long* out) {
  const std::string pat = std::string("\"") + key + "\"";
  size_t pos = text.find(pat);
  if (pos == std::string::npos) return false;
  pos = text.find(':', pos + pat.size());
  if (pos == std::string::npos) return false;
  char* end = nullptr;
  const long v = std::strtol(text.c_str() + pos + 1, &end, 10);
  if (end == text.c_str() + pos + 1) return false;
  *out = v;
  return true;
}
}  // namespace

void load_tune_table(bbp_plan p, const char* path) {
  FILE* fh = std::fopen(path, "rb");
  if (!fh) return;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), fh)) > 0) text.append(buf, got);
  std::fclose(fh);
  long v;
  if (read_int(text, "run", &v) && v >= 2 && v <= 4096 && v % 2 == 0) p->run = static_cast<int>(v);
  if (read_int(text, "streams", &v) && (v == 1 || v == 2)) p->streams = static_cast<int>(v);
  if (read_int(text, "grab", &v) && v >= 1 && v <= 1024) p->grab = static_cast<int>(v);
  if (read_int(text, "cta", &v) && v >= 32 && v <= 256 && v % 32 == 0) p->cta = static_cast<int>(v);
  if (read_int(text, "limb_bump", &v) && v >= 0 && v <= 2) p->limb_bump = static_cast<int>(v);
  if (read_int(text, "wide_min_bits", &v) && v >= kWideFloorBits && v <= kWideMinBits) p->wide_min_bits = static_cast<int>(v);
}

}  // namespace bbp
