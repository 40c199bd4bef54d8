// Text matrix loader and bicluster writer (host code).
//
// Input (arXiv 1807.09932, Methods, "Different input file formats support"): values separated by
// commas, tabs or semicolons; a header row of column names and a first column of row names are
// both optional, and when both are present the upper-left (corner) field may be missing, as R's
// write.table writes it. Missing values (Methods, "Handling missing values") are the empty field,
// NA / NaN, and a caller-chosen marker (for example 999 or 0), all read as NaN so that the
// evaluator's missing-value exclusion applies to them.
//
// Output (Methods, "Compatibility with R and Bioconductor"): the layout of the biclust package's
// bicluster result files: a title line, then per bicluster a line "rows cols" and a line each of
// row names and column names (columns in the bicluster's order).
//
// The file is read whole, split into lines, and the lines are parsed by several threads into a
// preallocated row-major float32 matrix.
#include <algorithm>
#include <charconv>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <string_view>
#include <thread>
#include <vector>

#include "ebic.h"
#include "ebic_internal.h"

namespace {

std::string_view trim(std::string_view s) {
  while (!s.empty() && (s.front() == ' ' || s.front() == '"' || s.front() == '\''))
    s.remove_prefix(1);
  while (!s.empty() &&
         (s.back() == ' ' || s.back() == '"' || s.back() == '\'' || s.back() == '\r'))
    s.remove_suffix(1);
  return s;
}

void split(std::string_view line, char delim, std::vector<std::string_view>* out) {
  out->clear();
  size_t start = 0;
  for (;;) {
    const size_t pos = line.find(delim, start);
    if (pos == std::string_view::npos) {
      out->push_back(trim(line.substr(start)));
      return;
    }
    out->push_back(trim(line.substr(start, pos - start)));
    start = pos + 1;
  }
}

bool parse_number(std::string_view s, double* v) {
  if (s.empty()) return false;
  if (s.front() == '+') s.remove_prefix(1);
  const char* b = s.data();
  const char* e = s.data() + s.size();
  auto r = std::from_chars(b, e, *v);
  return r.ec == std::errc() && r.ptr == e;
}

bool is_na(std::string_view s) {
  return s.empty() || s == "NA" || s == "NaN" || s == "nan" || s == "NAN" || s == "na";
}

struct Missing {
  bool has = false, numeric = false;
  double value = 0;
  std::string token;
};

// A data cell: true and *out set when it is a number or a missing value.
bool cell_value(std::string_view s, const Missing& mk, float* out) {
  if (mk.has && !mk.numeric && s == mk.token) {
    *out = std::numeric_limits<float>::quiet_NaN();
    return true;
  }
  if (is_na(s)) {
    *out = std::numeric_limits<float>::quiet_NaN();
    return true;
  }
  double v;
  if (!parse_number(s, &v)) return false;
  if (mk.has && mk.numeric && v == mk.value) v = std::numeric_limits<double>::quiet_NaN();
  *out = (float)v;
  return true;
}

char detect_delimiter(std::string_view first) {
  size_t best = 0;
  char d = ',';
  for (char c : {'\t', ';', ','}) {
    const size_t n = (size_t)std::count(first.begin(), first.end(), c);
    if (n > best) {
      best = n;
      d = c;
    }
  }
  return d;
}

char* dup(std::string_view s) {
  char* p = new char[s.size() + 1];
  std::memcpy(p, s.data(), s.size());
  p[s.size()] = '\0';
  return p;
}

}  // namespace

extern "C" {

int ebic_read_matrix_text(const char* path, char delimiter, const char* missing,
                          ebic_text_matrix** out) {
  using ebic::set_last_error;
  if (!path || !out) return set_last_error(EBIC_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (delimiter != 0 && delimiter != ',' && delimiter != '\t' && delimiter != ';')
    return set_last_error(EBIC_ERR_INVALID_ARG, "delimiter must be ',', '\\t', ';' or 0");
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_last_error(EBIC_ERR_INVALID_ARG, (std::string("cannot open ") + path).c_str());
  std::string buf;
  {
    char tmp[1 << 16];
    size_t n;
    while ((n = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.append(tmp, n);
    std::fclose(f);
  }
  // lines, skipping blank ones
  std::vector<std::string_view> lines;
  {
    std::string_view all(buf);
    size_t start = 0;
    while (start < all.size()) {
      size_t pos = all.find('\n', start);
      if (pos == std::string_view::npos) pos = all.size();
      std::string_view ln = all.substr(start, pos - start);
      if (!ln.empty() && ln.back() == '\r') ln.remove_suffix(1);
      if (!trim(ln).empty()) lines.push_back(ln);
      start = pos + 1;
    }
  }
  if (lines.empty()) return set_last_error(EBIC_ERR_INVALID_ARG, "the file has no data");
  const char d = delimiter ? delimiter : detect_delimiter(lines[0]);
  Missing mk;
  if (missing && *missing) {
    mk.has = true;
    mk.token = std::string(trim(missing));
    mk.numeric = parse_number(mk.token, &mk.value);
  }

  // layout (decided from the first two lines): the first line is a header row when it has one
  // field fewer than the second (R's layout without the corner field), when a field other than
  // its first is not a number, or when none of its fields is; a row-name column is present when
  // the first field of the first data row is not a number
  std::vector<std::string_view> f0, f1;
  split(lines[0], d, &f0);
  float tmpv;
  bool header = false;
  {
    std::vector<std::string_view> next;
    if (lines.size() > 1) split(lines[1], d, &next);
    size_t text = 0;
    bool text_after_first = false;
    for (size_t i = 0; i < f0.size(); ++i)
      if (!cell_value(f0[i], mk, &tmpv)) {
        ++text;
        if (i > 0) text_after_first = true;
      }
    header = (lines.size() > 1 && f0.size() + 1 == next.size()) || text_after_first ||
             text == f0.size();
  }
  size_t first_data = header ? 1 : 0;
  if (first_data >= lines.size()) return set_last_error(EBIC_ERR_INVALID_ARG, "no data rows");
  split(lines[first_data], d, &f1);
  const bool row_names = !f1.empty() && !cell_value(f1[0], mk, &tmpv);
  const size_t nfield = f1.size();
  const int64_t cols = (int64_t)nfield - (row_names ? 1 : 0);
  if (cols < 1 || cols > INT32_MAX) return set_last_error(EBIC_ERR_INVALID_ARG, "no data columns");
  std::vector<std::string_view> col_names;
  if (header) {
    if (f0.size() == (size_t)cols) {
      col_names = f0;  // no corner field (R's write.table layout) or no row names
    } else if (f0.size() == (size_t)cols + 1 && row_names) {
      col_names.assign(f0.begin() + 1, f0.end());  // corner field present
    } else {
      return set_last_error(EBIC_ERR_INVALID_ARG,
                            "the header has a different number of fields from the data rows");
    }
  }
  const int64_t rows = (int64_t)(lines.size() - first_data);

  auto* m = new ebic_text_matrix();
  m->rows = rows;
  m->cols = (int32_t)cols;
  m->values = new float[(size_t)rows * (size_t)cols];
  m->row_names = row_names ? new char*[rows]() : nullptr;
  m->col_names = header ? new char*[cols]() : nullptr;
  if (header)
    for (int64_t c = 0; c < cols; ++c) m->col_names[c] = dup(col_names[c]);

  // parse the rows in parallel; the first failure (lowest row) is reported
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const unsigned nt = (unsigned)std::min<int64_t>(hw, std::max<int64_t>(1, rows / 4096));
  std::vector<int64_t> bad_row(nt, -1);
  std::vector<int64_t> bad_col(nt, -1);
  auto work = [&](unsigned t) {
    std::vector<std::string_view> fs;
    const int64_t lo = rows * t / nt, hi = rows * (t + 1) / nt;
    for (int64_t r = lo; r < hi; ++r) {
      split(lines[first_data + r], d, &fs);
      if (fs.size() != nfield) {
        bad_row[t] = r;
        bad_col[t] = -1;
        return;
      }
      size_t k = 0;
      if (row_names) m->row_names[r] = dup(fs[k++]);
      float* dst = m->values + (size_t)r * (size_t)cols;
      for (int64_t c = 0; c < cols; ++c, ++k) {
        if (!cell_value(fs[k], mk, &dst[c])) {
          bad_row[t] = r;
          bad_col[t] = c;
          return;
        }
      }
    }
  };
  std::vector<std::thread> th;
  for (unsigned t = 1; t < nt; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& x : th) x.join();
  for (unsigned t = 0; t < nt; ++t) {
    if (bad_row[t] >= 0) {
      const int64_t line = bad_row[t] + (int64_t)first_data + 1;
      std::string msg = bad_col[t] < 0
                            ? "line " + std::to_string(line) + ": wrong number of fields"
                            : "line " + std::to_string(line) + ", column " +
                                  std::to_string(bad_col[t] + 1) + ": not a number";
      ebic_free_text_matrix(m);
      return set_last_error(EBIC_ERR_INVALID_ARG, msg.c_str());
    }
  }
  *out = m;
  return EBIC_OK;
}

int ebic_free_text_matrix(ebic_text_matrix* m) {
  if (!m) return EBIC_OK;
  if (m->row_names) {
    for (int64_t r = 0; r < m->rows; ++r) delete[] m->row_names[r];
    delete[] m->row_names;
  }
  if (m->col_names) {
    for (int32_t c = 0; c < m->cols; ++c) delete[] m->col_names[c];
    delete[] m->col_names;
  }
  delete[] m->values;
  delete m;
  return EBIC_OK;
}

int ebic_write_biclusters(const char* path, const char* title, const ebic_result* r,
                          const ebic_text_matrix* names) {
  using ebic::set_last_error;
  if (!path || !r) return set_last_error(EBIC_ERR_INVALID_ARG, "NULL argument");
  if (r->n > 0 && !r->bitmaps)
    return set_last_error(EBIC_ERR_INVALID_ARG, "the result carries no row bitmaps");
  if (names && (names->rows + 31) / 32 != r->words)
    return set_last_error(EBIC_ERR_INVALID_ARG, "names are for a matrix of another size");
  FILE* f = std::fopen(path, "w");
  if (!f) return set_last_error(EBIC_ERR_INVALID_ARG, (std::string("cannot create ") + path).c_str());
  std::fprintf(f, "%s\n", title ? title : "EBIC");
  for (uint32_t b = 0; b < r->n; ++b) {
    const uint32_t o = r->offsets[b], L = r->offsets[b + 1] - o;
    const uint32_t* bm = r->bitmaps + (size_t)b * (size_t)r->words;
    std::vector<int64_t> rws;
    for (int64_t w = 0; w < r->words; ++w)
      for (uint32_t x = bm[w]; x; x &= x - 1) rws.push_back(w * 32 + __builtin_ctz(x));
    std::fprintf(f, "%zu %u\n", rws.size(), L);
    for (size_t i = 0; i < rws.size(); ++i) {
      if (i) std::fputc(' ', f);
      if (names && names->row_names)
        std::fputs(names->row_names[rws[i]], f);
      else
        std::fprintf(f, "%lld", (long long)rws[i] + 1);
    }
    std::fputc('\n', f);
    for (uint32_t j = 0; j < L; ++j) {
      if (j) std::fputc(' ', f);
      const uint32_t c = r->cols[o + j];
      if (names && names->col_names && (int32_t)c < names->cols)
        std::fputs(names->col_names[c], f);
      else
        std::fprintf(f, "%u", c + 1);
    }
    std::fputc('\n', f);
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? EBIC_OK : set_last_error(EBIC_ERR_INVALID_ARG, "write failed");
}

}  // extern "C"
