// Model files (Sec. 3.1, reading and writing IMDPs): the PRISM explicit files
// (.sta, .lab, .tra, .pctl) and the bmdp-tool format, read into and written from
// the CSC arrays that imdp_create_csc takes. Host code only: no CUDA call here.
//
// The paper names the formats and what each carries (PRISM: states, labels,
// interval transitions and the property in four files; bmdp-tool: source,
// action, destination and bounds per line plus the terminal states, no horizon
// or modes) without a byte-level layout; the layouts read and written here are
// the ones include/imdp.h states.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <algorithm>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "imdp_internal.h"

using namespace imdp;

namespace {

constexpr double kDefaultEps = 1e-6;  // infinite-time properties: the files carry no tolerance

// One stored transition as read from a file, with the line it came from.
struct Entry {
  int32_t s, a, d;
  int32_t line;
  double lo, up;
};

bool read_text(const std::string& path, std::string* out) {
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return false;
  std::string s;
  std::vector<char> buf(1 << 16);
  size_t n;
  while ((n = std::fread(buf.data(), 1, buf.size(), f)) > 0) s.append(buf.data(), n);
  const bool ok = !std::ferror(f);
  std::fclose(f);
  if (ok) *out = std::move(s);
  return ok;
}

// Whitespace-separated tokens of an ASCII file, with line numbers for errors.
// The text is a std::string, so strtoll / strtod always meet a terminating NUL.
class Lexer {
 public:
  Lexer(const std::string& text, std::string name)
      : p_(text.c_str()), end_(text.c_str() + text.size()), name_(std::move(name)) {}
  // The part [begin, end) of a NUL-terminated text, whose first line is `line`.
  Lexer(const char* begin, const char* end, std::string name, int64_t line)
      : p_(begin), end_(end), name_(std::move(name)), line_(line) {}

  // Skip blanks; newlines too when `lines`.
  void skip(bool lines) {
    while (p_ < end_) {
      const char c = *p_;
      if (c == '\n') {
        if (!lines) return;
        ++line_;
        ++p_;
      } else if (c == ' ' || c == '\t' || c == '\r') {
        ++p_;
      } else {
        return;
      }
    }
  }
  bool at_end() {
    skip(true);
    return p_ >= end_;
  }
  bool at_eol() {
    skip(false);
    return p_ >= end_ || *p_ == '\n';
  }
  // Drop what is left of the current line.
  void next_line() {
    while (p_ < end_ && *p_ != '\n') ++p_;
  }
  // An integer token; with `term` it must be followed directly by that
  // character, which is consumed too ("3:" in .sta / .lab, "0=" in .lab).
  bool integer(int64_t* v, bool lines = true, char term = '\0') {
    skip(lines);
    if (p_ >= end_ || *p_ == '\n') return false;
    char* e = nullptr;
    const long long x = std::strtoll(p_, &e, 10);
    if (e == p_) return false;
    if (term) {
      if (e >= end_ || *e != term) return false;
      ++e;
    } else if (!ends_token(e)) {
      return false;
    }
    p_ = e;
    *v = x;
    return true;
  }
  bool number(double* v, bool lines = true) {
    skip(lines);
    if (p_ >= end_ || *p_ == '\n') return false;
    char* e = nullptr;
    const double x = std::strtod(p_, &e);
    if (e == p_ || !ends_token(e)) return false;
    p_ = e;
    *v = x;
    return true;
  }
  // "[lower,upper]" (blanks allowed inside) or a plain probability p = [p, p].
  bool interval(double* lo, double* up) {
    skip(false);
    if (p_ < end_ && *p_ == '[') {
      ++p_;
      if (!bare_number(lo) || !expect(',') || !bare_number(up) || !expect(']') || !ends_token(p_)) return false;
      return true;
    }
    if (!number(lo, false)) return false;
    *up = *lo;
    return true;
  }
  // Consume character `c` after optional blanks on the same line.
  bool expect(char c) {
    skip(false);
    if (p_ < end_ && *p_ == c) {
      ++p_;
      return true;
    }
    return false;
  }
  // Characters up to (not including) `stop` on the current line.
  bool until(char stop, std::string* out) {
    const char* b = p_;
    while (p_ < end_ && *p_ != stop && *p_ != '\n') ++p_;
    if (p_ >= end_ || *p_ != stop) return false;
    out->assign(b, p_);
    ++p_;
    return true;
  }
  char peek() {
    skip(false);
    return p_ < end_ ? *p_ : '\0';
  }
  std::string where() const { return name_ + ":" + std::to_string(line_); }
  int64_t line64() const { return line_; }
  const char* pos() const { return p_; }

 private:
  bool ends_token(const char* e) const {
    return e >= end_ || *e == ' ' || *e == '\t' || *e == '\r' || *e == '\n';
  }
  bool bare_number(double* v) {
    skip(false);
    if (p_ >= end_ || *p_ == '\n') return false;
    char* e = nullptr;
    const double x = std::strtod(p_, &e);
    if (e == p_) return false;
    p_ = e;
    *v = x;
    return true;
  }
  const char* p_;
  const char* end_;
  std::string name_;
  int64_t line_ = 1;
};

imdp_status parse_error(const std::string& where, const std::string& what) {
  set_error(where + ": " + what);
  return IMDP_EINVAL;
}

template <class T>
T* copy_out(const std::vector<T>& v) {
  T* p = static_cast<T*>(std::malloc(sizeof(T) * std::max<size_t>(v.size(), 1)));
  if (p && !v.empty()) std::memcpy(p, v.data(), sizeof(T) * v.size());
  return p;
}

void free_file(imdp_file* f) {
  if (!f) return;
  std::free(f->stateptr);
  std::free(f->colptr);
  std::free(f->rowval);
  std::free(f->lower);
  std::free(f->upper);
  std::free(f->action);
  std::free(const_cast<int32_t*>(f->spec.reach));
  std::free(const_cast<int32_t*>(f->spec.avoid));
  std::free(f);
}

// Sort the entries into CSC order (state, action, destination), check that no
// transition repeats and, for PRISM, that each state's choices are 0, 1, ...;
// give a state without transitions one absorbing column; copy the arrays out.
imdp_status assemble(const std::string& name, int32_t n, std::vector<Entry>& es, bool dense_choices,
                     std::vector<int32_t> reach, std::vector<int32_t> avoid, const imdp_spec& spec, imdp_file** out) {
  const auto csc_order = [](const Entry& x, const Entry& y) {
    if (x.s != y.s) return x.s < y.s;
    if (x.a != y.a) return x.a < y.a;
    return x.d < y.d;
  };
  if (!std::is_sorted(es.begin(), es.end(), csc_order)) std::sort(es.begin(), es.end(), csc_order);
  std::vector<int32_t> sp, cp, rv, act;
  std::vector<double> lo, up;
  sp.reserve((size_t)n + 1);
  rv.reserve(es.size() + (size_t)n);
  lo.reserve(es.size() + (size_t)n);
  up.reserve(es.size() + (size_t)n);
  sp.push_back(0);
  cp.push_back(0);
  size_t i = 0;
  for (int32_t s = 0; s < n; ++s) {
    if (i >= es.size() || es[i].s != s) {
      // no transition: absorbing
      rv.push_back(s);
      lo.push_back(1.0);
      up.push_back(1.0);
      act.push_back(-1);
      cp.push_back((int32_t)rv.size());
    }
    int32_t next_choice = 0;
    while (i < es.size() && es[i].s == s) {
      const int32_t a = es[i].a;
      if (dense_choices && a != next_choice)
        return parse_error(name + ":" + std::to_string(es[i].line),
                           "state " + std::to_string(s) + " has choice " + std::to_string(a) + " but no choice " +
                               std::to_string(next_choice));
      ++next_choice;
      for (; i < es.size() && es[i].s == s && es[i].a == a; ++i) {
        if (!rv.empty() && (int32_t)rv.size() > cp.back() && rv.back() == es[i].d)
          return parse_error(name + ":" + std::to_string(es[i].line),
                             "duplicate transition " + std::to_string(s) + " " + std::to_string(a) + " " +
                                 std::to_string(es[i].d));
        rv.push_back(es[i].d);
        lo.push_back(es[i].lo);
        up.push_back(es[i].up);
      }
      if (rv.size() > (size_t)INT32_MAX - 1) return parse_error(name, "more than 2^31 - 1 transitions");
      act.push_back(a);
      cp.push_back((int32_t)rv.size());
    }
    if (cp.size() > (size_t)INT32_MAX) return parse_error(name, "more than 2^31 - 1 state-action pairs");
    sp.push_back((int32_t)cp.size() - 1);
  }
  std::sort(reach.begin(), reach.end());
  reach.erase(std::unique(reach.begin(), reach.end()), reach.end());
  std::sort(avoid.begin(), avoid.end());
  avoid.erase(std::unique(avoid.begin(), avoid.end()), avoid.end());

  imdp_file* f = static_cast<imdp_file*>(std::calloc(1, sizeof(imdp_file)));
  if (!f) {
    set_error("host allocation failed");
    return IMDP_ENOMEM;
  }
  f->n_states = n;
  f->n_cols = (int32_t)cp.size() - 1;
  f->nnz = (int64_t)rv.size();
  f->stateptr = copy_out(sp);
  f->colptr = copy_out(cp);
  f->rowval = copy_out(rv);
  f->lower = copy_out(lo);
  f->upper = copy_out(up);
  f->action = copy_out(act);
  f->spec = spec;
  f->spec.reach = copy_out(reach);
  f->spec.n_reach = (int32_t)reach.size();
  f->spec.avoid = copy_out(avoid);
  f->spec.n_avoid = (int32_t)avoid.size();
  if (!f->stateptr || !f->colptr || !f->rowval || !f->lower || !f->upper || !f->action || !f->spec.reach ||
      !f->spec.avoid) {
    free_file(f);
    set_error("host allocation failed");
    return IMDP_ENOMEM;
  }
  *out = f;
  return IMDP_OK;
}

imdp_spec default_spec() {
  imdp_spec s;
  std::memset(&s, 0, sizeof(s));
  s.property = IMDP_REACH;
  s.infinite_time = 0;
  s.horizon = 0;
  s.eps = kDefaultEps;
  s.pessimistic = 1;
  s.maximize = 1;
  s.discount = 1.0;
  return s;
}

bool finite_bounds(double lo, double up) { return std::isfinite(lo) && std::isfinite(up); }

// Structure of host CSC arrays given to a writer (the checks of imdp_create_csc
// that do not concern the bound values).
imdp_status check_host_csc(int32_t n, int32_t m, const int32_t* sp, const int32_t* cp, const int32_t* rv,
                           const double* lo, const double* up) {
  if (n < 1 || m < n || !sp || !cp || !rv || !lo || !up) {
    set_error("need n_states >= 1, n_cols >= n_states and non-NULL arrays");
    return IMDP_EINVAL;
  }
  if (sp[0] != 0 || sp[n] != m || cp[0] != 0) {
    set_error("stateptr must run from 0 to n_cols and colptr start at 0");
    return IMDP_EINVAL;
  }
  for (int32_t s = 0; s < n; ++s)
    if (sp[s + 1] <= sp[s]) {
      set_error("every state needs at least one column (stateptr strictly increasing)");
      return IMDP_EINVAL;
    }
  for (int32_t j = 0; j < m; ++j) {
    if (cp[j + 1] <= cp[j]) {
      set_error("every column needs at least one transition (colptr strictly increasing)");
      return IMDP_EINVAL;
    }
    for (int32_t e = cp[j]; e < cp[j + 1]; ++e)
      if (rv[e] < 0 || rv[e] >= n || (e > cp[j] && rv[e] <= rv[e - 1])) {
        set_error("rowval out of range or not strictly increasing in column " + std::to_string(j));
        return IMDP_EINVAL;
      }
  }
  return IMDP_OK;
}

// fprintf into a file, remembering whether any write failed.
struct Out {
  FILE* f = nullptr;
  bool ok = true;
  explicit Out(const std::string& path) : f(std::fopen(path.c_str(), "w")) { ok = f != nullptr; }
  ~Out() {
    if (f) std::fclose(f);
  }
  template <class... A>
  void print(const char* fmt, A... a) {
    if (ok && std::fprintf(f, fmt, a...) < 0) ok = false;
  }
  void put(const char* text) {
    if (ok && std::fputs(text, f) < 0) ok = false;
  }
  void write(const std::string& text) {
    if (ok && !text.empty() && std::fwrite(text.data(), 1, text.size(), f) != text.size()) ok = false;
  }
  bool close() {
    if (f && std::fclose(f) != 0) ok = false;
    f = nullptr;
    return ok;
  }
};

// ---------------------------------------------------------------- host threads
//
// Reading and writing large models is bound by number parsing and formatting
// (strtod / snprintf, a few hundred ns per bound), so both run on all host
// cores: the text is cut at line starts into one part per thread, and the
// parts are joined in file order.

unsigned host_threads(size_t bytes) {
  if (bytes < ((size_t)1 << 20)) return 1;  // small files: not worth a thread
  const unsigned hc = std::thread::hardware_concurrency();
  return std::max(1u, std::min(hc ? hc : 1u, 16u));
}

// f(i) for i in [0, n), on up to n threads; f must not throw. A thread that
// cannot be started runs its part on the calling thread.
template <class F>
void run_parts(unsigned n, F&& f) {
  std::vector<std::thread> th;
  for (unsigned i = 1; i < n; ++i) {
    try {
      th.emplace_back(f, i);
    } catch (...) {
      f(i);
    }
  }
  f(0);
  for (auto& t : th) t.join();
}

// Parse the entry lines of [body, end of text) with `one` (reads one entry from a
// lexer standing on its first token, or sets a message and returns false). The
// first error in file order is reported with its line in the whole file; the
// entries come back in file order. `body_line` is the line `body` lies on.
template <class One>
imdp_status parse_body(const std::string& text, const char* body, int64_t body_line, const std::string& name,
                       One one, std::vector<Entry>* out) {
  const char* end = text.c_str() + text.size();
  const unsigned T = host_threads((size_t)(end - body));
  std::vector<const char*> cut(T + 1);
  cut[0] = body;
  cut[T] = end;
  for (unsigned i = 1; i < T; ++i) {
    const char* c = std::max(cut[i - 1], body + (size_t)(end - body) * i / T);
    const char* nl = static_cast<const char*>(std::memchr(c, '\n', (size_t)(end - c)));
    cut[i] = nl ? nl + 1 : end;
  }
  struct Part {
    std::vector<Entry> es;
    int64_t newlines = 0;
    bool bad = false, oom = false;
    int64_t bad_line = 0;
    std::string msg;
  };
  std::vector<Part> parts(T);
  run_parts(T, [&](unsigned i) {
    Part& P = parts[i];
    try {
      Lexer lx(cut[i], cut[i + 1], name, 1);
      while (!lx.at_end()) {
        Entry e{};
        const int64_t ln = lx.line64();
        if (!one(lx, &e, &P.msg)) {
          P.bad = true;
          P.bad_line = lx.line64();
          return;
        }
        e.line = (int32_t)std::min<int64_t>(ln, INT32_MAX);  // local for now
        P.es.push_back(e);
      }
      P.newlines = lx.line64() - 1;
    } catch (...) {
      P.bad = P.oom = true;
    }
  });
  int64_t base = body_line;  // line of each part's first character
  size_t total = 0;
  for (unsigned i = 0; i < T; ++i) {
    Part& P = parts[i];
    if (P.oom) throw std::bad_alloc();
    if (P.bad) return parse_error(name + ":" + std::to_string(base + P.bad_line - 1), P.msg);
    for (Entry& e : P.es) e.line = (int32_t)std::min<int64_t>(base + e.line - 1, INT32_MAX);
    base += P.newlines;
    total += P.es.size();
  }
  out->clear();
  out->reserve(total);
  for (Part& P : parts) {
    out->insert(out->end(), P.es.begin(), P.es.end());
    std::vector<Entry>().swap(P.es);
  }
  return IMDP_OK;
}

// Write one line per stored transition, `fmt(buf, cap, s, action, e)` giving the
// text of entry e (column action of state s). States are taken in blocks of
// about kBlockEntries entries; the blocks of a round are formatted in parallel
// and written in order.
constexpr int64_t kBlockEntries = 1 << 18;

template <class Fmt>
void write_entry_lines(Out& o, int32_t n, const int32_t* sp, const int32_t* cp, Fmt fmt) {
  std::vector<int32_t> starts{0};
  int64_t acc = 0;
  for (int32_t s = 0; s < n; ++s) {
    acc += cp[sp[s + 1]] - cp[sp[s]];
    if (acc >= kBlockEntries) {
      starts.push_back(s + 1);
      acc = 0;
    }
  }
  if (starts.back() != n) starts.push_back(n);
  const size_t blocks = starts.size() - 1;
  const unsigned T = host_threads((size_t)cp[sp[n]] * 40);
  for (size_t w = 0; w < blocks && o.ok; w += T) {
    const unsigned wn = (unsigned)std::min<size_t>(T, blocks - w);
    std::vector<std::string> bufs(wn);
    std::vector<char> failed(wn, 0);
    run_parts(wn, [&](unsigned b) {
      try {
        std::string& text = bufs[b];
        char line[160];
        for (int32_t s = starts[w + b]; s < starts[w + b + 1]; ++s)
          for (int32_t j = sp[s]; j < sp[s + 1]; ++j)
            for (int32_t e = cp[j]; e < cp[j + 1]; ++e) {
              const int k = fmt(line, sizeof(line), s, j - sp[s], e);
              if (k > 0) text.append(line, (size_t)std::min<int>(k, (int)sizeof(line) - 1));
            }
      } catch (...) {
        failed[b] = 1;
      }
    });
    for (unsigned b = 0; b < wn; ++b) {
      if (failed[b]) throw std::bad_alloc();
      o.write(bufs[b]);
    }
  }
}

imdp_status io_error(const std::string& path) {
  set_error("cannot write " + path);
  return IMDP_EIO;
}

// ---------------------------------------------------------------- PRISM property

// P<strategy>[<adversary>]=? [ F[<=K] "goal" ] or [ !"avoid" U[<=K] "goal" ], blanks
// anywhere outside the quoted labels.
imdp_status parse_property(const std::string& where, const std::string& text, imdp_spec* spec, std::string* goal,
                           std::string* avoid) {
  std::string q;  // the property with blanks outside quotes removed
  bool quoted = false;
  for (char c : text) {
    if (c == '"') quoted = !quoted;
    if (quoted || !(c == ' ' || c == '\t' || c == '\r' || c == '\n')) q.push_back(c);
  }
  size_t i = 0;
  auto take = [&](const char* lit) {
    const size_t n = std::strlen(lit);
    if (q.compare(i, n, lit) == 0) {
      i += n;
      return true;
    }
    return false;
  };
  auto label = [&](std::string* out) {
    if (!take("\"")) return false;
    const size_t e = q.find('"', i);
    if (e == std::string::npos || e == i) return false;
    out->assign(q, i, e - i);
    i = e + 1;
    return true;
  };
  auto bound = [&]() -> bool {
    if (!take("<=")) {
      spec->infinite_time = 1;
      spec->horizon = 0;
      return true;
    }
    size_t e = i;
    while (e < q.size() && q[e] >= '0' && q[e] <= '9') ++e;
    if (e == i || e - i > 9) return false;
    spec->infinite_time = 0;
    spec->horizon = std::atoi(q.substr(i, e - i).c_str());
    i = e;
    return true;
  };
  if (q.compare(0, 1, "R") == 0)
    return parse_error(where, "reward properties cannot be read from PRISM explicit files (no reward file)");
  if (!take("P")) return parse_error(where, "expected a P...=? [ ... ] property");
  if (take("max"))
    spec->maximize = 1;
  else if (take("min"))
    spec->maximize = 0;
  else
    return parse_error(where, "expected Pmax or Pmin");
  if (take("max"))
    spec->pessimistic = 0;
  else if (take("min"))
    spec->pessimistic = 1;
  else
    spec->pessimistic = 1;  // no adversary given: the robust (pessimistic) reading
  if (!take("=?") || !take("[")) return parse_error(where, "expected =? [");
  if (take("(!")) {
    if (!label(avoid) || !take(")")) return parse_error(where, "expected (!\"label\")");
  } else if (take("!")) {
    if (!label(avoid)) return parse_error(where, "expected !\"label\"");
  }
  if (!avoid->empty()) {
    if (!take("U")) return parse_error(where, "expected U after the avoided label");
    spec->property = IMDP_REACH_AVOID;
  } else {
    if (!take("F")) return parse_error(where, "expected F or !\"label\" U");
    spec->property = IMDP_REACH;
  }
  if (!bound()) return parse_error(where, "expected <=K with K a nonnegative integer");
  if (!label(goal)) return parse_error(where, "expected the target \"label\"");
  if (!take("]") || i != q.size()) return parse_error(where, "expected ] at the end of the property");
  return IMDP_OK;
}

// Allocation failures (and any other exception) become a status: nothing is
// thrown across the C ABI.
template <class F>
imdp_status guarded(F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return IMDP_ENOMEM;
  } catch (const std::exception& e) {
    set_error(e.what());
    return IMDP_EINVAL;
  }
}

}  // namespace

extern "C" {

IMDP_API void imdp_file_free(imdp_file* f) { free_file(f); }

IMDP_API imdp_status imdp_read_bmdp_tool(const char* path, imdp_file** out) {
  return guarded([&]() -> imdp_status {
    set_error("");
    if (!path || !out) {
      set_error("NULL path or out");
      return IMDP_EINVAL;
    }
    *out = nullptr;
    std::string text;
    if (!read_text(path, &text)) {
      set_error(std::string("cannot read ") + path);
      return IMDP_EIO;
    }
    Lexer lx(text, path);
    int64_t n = 0, na = 0, nt = 0;
    if (!lx.integer(&n) || n < 1 || n >= INT32_MAX) return parse_error(lx.where(), "expected the number of states (>= 1)");
    if (!lx.integer(&na) || na < 1 || na >= INT32_MAX)
      return parse_error(lx.where(), "expected the number of actions (>= 1)");
    if (!lx.integer(&nt) || nt < 0 || nt > n)
      return parse_error(lx.where(), "expected the number of terminal states (0 .. n_states)");
    std::vector<int32_t> term((size_t)nt);
    for (int64_t i = 0; i < nt; ++i) {
      int64_t t = -1;
      if (!lx.integer(&t) || t < 0 || t >= n) return parse_error(lx.where(), "expected a terminal state in [0, n_states)");
      term[(size_t)i] = (int32_t)t;
    }
    std::vector<Entry> es;
    imdp_status st = parse_body(text, lx.pos(), lx.line64(), path, [&](Lexer& l, Entry* e, std::string* msg) {
      int64_t s = -1, a = -1, d = -1;
      double lo = 0, up = 0;
      if (!l.integer(&s) || !l.integer(&a, false) || !l.integer(&d, false) || !l.number(&lo, false) ||
          !l.number(&up, false) || !l.at_eol()) {
        *msg = "expected: source action destination lower upper";
        return false;
      }
      if (s < 0 || s >= n || d < 0 || d >= n) {
        *msg = "state index out of range";
        return false;
      }
      if (a < 0 || a >= na) {
        *msg = "action index out of range [0, n_actions)";
        return false;
      }
      if (!finite_bounds(lo, up)) {
        *msg = "bounds must be finite numbers";
        return false;
      }
      *e = Entry{(int32_t)s, (int32_t)a, (int32_t)d, 0, lo, up};
      return true;
    }, &es);
    if (st != IMDP_OK) return st;
    imdp_spec spec = default_spec();
    return assemble(path, (int32_t)n, es, false, std::move(term), {}, spec, out);
  });
}

IMDP_API imdp_status imdp_write_bmdp_tool(const char* path, int32_t n_states, int32_t n_cols, const int32_t* stateptr,
                                          const int32_t* colptr, const int32_t* rowval, const double* lower,
                                          const double* upper, const int32_t* terminal, int32_t n_terminal) {
  return guarded([&]() -> imdp_status {
    set_error("");
    if (!path) {
      set_error("NULL path");
      return IMDP_EINVAL;
    }
    imdp_status st = check_host_csc(n_states, n_cols, stateptr, colptr, rowval, lower, upper);
    if (st != IMDP_OK) return st;
    if (n_terminal < 0 || (n_terminal > 0 && !terminal)) {
      set_error("terminal states: need n_terminal >= 0 and a non-NULL array");
      return IMDP_EINVAL;
    }
    for (int32_t i = 0; i < n_terminal; ++i)
      if (terminal[i] < 0 || terminal[i] >= n_states) {
        set_error("terminal state out of range");
        return IMDP_EINVAL;
      }
    int32_t na = 1;
    for (int32_t s = 0; s < n_states; ++s) na = std::max(na, stateptr[s + 1] - stateptr[s]);
    Out o(path);
    o.print("%d\n%d\n%d\n", n_states, na, n_terminal);
    for (int32_t i = 0; i < n_terminal; ++i) o.print("%d\n", terminal[i]);
    write_entry_lines(o, n_states, stateptr, colptr, [&](char* buf, size_t cap, int32_t s, int32_t a, int32_t e) {
      return std::snprintf(buf, cap, "%d %d %d %.17g %.17g\n", s, a, rowval[e], lower[e], upper[e]);
    });
    return o.close() ? IMDP_OK : io_error(path);
  });
}

IMDP_API imdp_status imdp_read_prism(const char* path_stem, imdp_file** out) {
  return guarded([&]() -> imdp_status {
    set_error("");
    if (!path_stem || !out) {
      set_error("NULL path or out");
      return IMDP_EINVAL;
    }
    *out = nullptr;
    const std::string stem = path_stem;
    std::string tra, sta, lab, pctl;
    for (auto& pr : {std::make_pair(".tra", &tra), std::make_pair(".sta", &sta), std::make_pair(".lab", &lab),
                     std::make_pair(".pctl", &pctl)})
      if (!read_text(stem + pr.first, pr.second)) {
        set_error("cannot read " + stem + pr.first);
        return IMDP_EIO;
      }

    // .tra: header, then one interval transition per line
    Lexer lt(tra, stem + ".tra");
    int64_t n = 0, m = 0, t = 0;
    if (!lt.integer(&n) || n < 1 || n >= INT32_MAX || !lt.integer(&m, false) || m < 0 || m >= INT32_MAX ||
        !lt.integer(&t, false) || t < 0 || t >= INT32_MAX || !lt.at_eol())
      return parse_error(lt.where(), "expected: n_states n_choices n_transitions");
    std::vector<Entry> es;
    imdp_status pst = parse_body(tra, lt.pos(), lt.line64(), stem + ".tra", [&](Lexer& l, Entry* e, std::string* msg) {
      int64_t s = -1, c = -1, d = -1;
      double lo = 0, up = 0;
      if (!l.integer(&s) || !l.integer(&c, false) || !l.integer(&d, false) || !l.interval(&lo, &up)) {
        *msg = "expected: source choice destination [lower,upper]";
        return false;
      }
      l.next_line();  // an action name may follow
      if (s < 0 || s >= n || d < 0 || d >= n) {
        *msg = "state index out of range";
        return false;
      }
      if (c < 0 || c >= std::max<int64_t>(m, 1)) {
        *msg = "choice index out of range";
        return false;
      }
      if (!finite_bounds(lo, up)) {
        *msg = "bounds must be finite numbers";
        return false;
      }
      *e = Entry{(int32_t)s, (int32_t)c, (int32_t)d, 0, lo, up};
      return true;
    }, &es);
    if (pst != IMDP_OK) return pst;
    if ((int64_t)es.size() != t)
      return parse_error(stem + ".tra", "header gives " + std::to_string(t) + " transitions, the file has " +
                                            std::to_string(es.size()));
    {
      // the number of (state, choice) pairs must match the header
      std::vector<std::pair<int32_t, int32_t>> sc(es.size());
      for (size_t i = 0; i < es.size(); ++i) sc[i] = {es[i].s, es[i].a};
      std::sort(sc.begin(), sc.end());
      const int64_t pairs = (int64_t)(std::unique(sc.begin(), sc.end()) - sc.begin());
      if (pairs != m)
        return parse_error(stem + ".tra", "header gives " + std::to_string(m) + " choices, the file has " +
                                              std::to_string(pairs));
    }

    // .sta: "(vars)" then "i:(values)" for every state
    {
      Lexer ls(sta, stem + ".sta");
      if (ls.at_end() || ls.peek() != '(') return parse_error(ls.where(), "expected the variable list \"(...)\"");
      ls.next_line();
      std::vector<char> seen((size_t)n, 0);
      int64_t count = 0;
      while (!ls.at_end()) {
        int64_t i = -1;
        if (!ls.integer(&i, true, ':') || ls.peek() != '(') return parse_error(ls.where(), "expected i:(values)");
        if (i < 0 || i >= n || seen[(size_t)i]) return parse_error(ls.where(), "state index out of range or repeated");
        seen[(size_t)i] = 1;
        ++count;
        ls.next_line();
      }
      if (count != n)
        return parse_error(stem + ".sta", "lists " + std::to_string(count) + " states, .tra has " + std::to_string(n));
    }

    // .lab: id="name" pairs, then "s: id id ..." lines
    std::map<std::string, std::vector<int32_t>> labelled;
    {
      Lexer ll(lab, stem + ".lab");
      std::map<int64_t, std::string> names;
      while (!ll.at_eol()) {
        int64_t id = -1;
        std::string name;
        if (!ll.integer(&id, false, '=') || !ll.expect('"') || !ll.until('"', &name) || name.empty())
          return parse_error(ll.where(), "expected id=\"name\" pairs on the first line");
        if (!names.emplace(id, name).second) return parse_error(ll.where(), "label id repeated");
        labelled[name];
      }
      while (!ll.at_end()) {
        int64_t s = -1;
        if (!ll.integer(&s, true, ':')) return parse_error(ll.where(), "expected s: id id ...");
        if (s < 0 || s >= n) return parse_error(ll.where(), "state index out of range");
        while (!ll.at_eol()) {
          int64_t id = -1;
          if (!ll.integer(&id, false)) return parse_error(ll.where(), "expected a label id");
          const auto it = names.find(id);
          if (it == names.end()) return parse_error(ll.where(), "label id not declared on the first line");
          labelled[it->second].push_back((int32_t)s);
        }
      }
    }

    // .pctl: the first line that is neither blank nor a // comment
    imdp_spec spec = default_spec();
    std::string goal, avoid;
    {
      size_t b = 0;
      int32_t line = 0;
      std::string prop;
      while (b < pctl.size()) {
        size_t e = pctl.find('\n', b);
        if (e == std::string::npos) e = pctl.size();
        ++line;
        const std::string l = pctl.substr(b, e - b);
        b = e + 1;
        const size_t f = l.find_first_not_of(" \t\r");
        if (f == std::string::npos || l.compare(f, 2, "//") == 0) continue;
        prop = l;
        break;
      }
      const std::string where = stem + ".pctl:" + std::to_string(line);
      if (prop.empty()) return parse_error(stem + ".pctl", "no property");
      imdp_status st = parse_property(where, prop, &spec, &goal, &avoid);
      if (st != IMDP_OK) return st;
      if (!labelled.count(goal)) return parse_error(where, "label \"" + goal + "\" is not in .lab");
      if (!avoid.empty() && !labelled.count(avoid)) return parse_error(where, "label \"" + avoid + "\" is not in .lab");
    }
    std::vector<int32_t> reach = labelled[goal];
    std::vector<int32_t> av = avoid.empty() ? std::vector<int32_t>() : labelled[avoid];
    return assemble(stem + ".tra", (int32_t)n, es, true, std::move(reach), std::move(av), spec, out);
  });
}

IMDP_API imdp_status imdp_write_prism(const char* path_stem, int32_t n_states, int32_t n_cols, const int32_t* stateptr,
                                      const int32_t* colptr, const int32_t* rowval, const double* lower,
                                      const double* upper, const imdp_spec* spec) {
  return guarded([&]() -> imdp_status {
    set_error("");
    if (!path_stem || !spec) {
      set_error("NULL path or spec");
      return IMDP_EINVAL;
    }
    imdp_status st = check_host_csc(n_states, n_cols, stateptr, colptr, rowval, lower, upper);
    if (st != IMDP_OK) return st;
    if (spec->property != IMDP_REACH && spec->property != IMDP_REACH_AVOID) {
      set_error("only reachability and reach-avoid properties can be written as PRISM explicit files");
      return IMDP_EINVAL;
    }
    const bool ra = spec->property == IMDP_REACH_AVOID;
    if (spec->n_reach < 0 || (spec->n_reach > 0 && !spec->reach) || (ra && (spec->n_avoid < 0 ||
                                                                            (spec->n_avoid > 0 && !spec->avoid)))) {
      set_error("reach / avoid sets: need counts >= 0 and non-NULL arrays");
      return IMDP_EINVAL;
    }
    if (!spec->infinite_time && spec->horizon < 0) {
      set_error("horizon must be >= 0");
      return IMDP_EINVAL;
    }
    std::vector<uint8_t> mark((size_t)n_states, 0);  // bit 0: reach, bit 1: avoid
    for (int32_t i = 0; i < spec->n_reach; ++i) {
      if (spec->reach[i] < 0 || spec->reach[i] >= n_states) {
        set_error("reach state out of range");
        return IMDP_EINVAL;
      }
      mark[spec->reach[i]] |= 1;
    }
    for (int32_t i = 0; ra && i < spec->n_avoid; ++i) {
      if (spec->avoid[i] < 0 || spec->avoid[i] >= n_states) {
        set_error("avoid state out of range");
        return IMDP_EINVAL;
      }
      mark[spec->avoid[i]] |= 2;
    }
    const std::string stem = path_stem;
    {
      Out o(stem + ".sta");
      o.put("(s)\n");
      for (int32_t s = 0; s < n_states; ++s) o.print("%d:(%d)\n", s, s);
      if (!o.close()) return io_error(stem + ".sta");
    }
    {
      Out o(stem + ".lab");
      o.print("0=\"init\" 1=\"deadlock\" 2=\"reach\"%s\n", ra ? " 3=\"avoid\"" : "");
      for (int32_t s = 0; s < n_states; ++s) {
        if (s != 0 && !mark[s]) continue;
        o.print("%d:", s);
        if (s == 0) o.put(" 0");
        if (mark[s] & 1) o.put(" 2");
        if (mark[s] & 2) o.put(" 3");
        o.put("\n");
      }
      if (!o.close()) return io_error(stem + ".lab");
    }
    {
      Out o(stem + ".tra");
      o.print("%d %d %d\n", n_states, n_cols, colptr[n_cols]);
      write_entry_lines(o, n_states, stateptr, colptr, [&](char* buf, size_t cap, int32_t s, int32_t c, int32_t e) {
        return std::snprintf(buf, cap, "%d %d %d [%.17g,%.17g]\n", s, c, rowval[e], lower[e], upper[e]);
      });
      if (!o.close()) return io_error(stem + ".tra");
    }
    {
      Out o(stem + ".pctl");
      const char* strat = spec->maximize ? "max" : "min";
      const char* adv = spec->pessimistic ? "min" : "max";
      const std::string bound = spec->infinite_time ? std::string() : "<=" + std::to_string(spec->horizon);
      if (ra)
        o.print("P%s%s=? [ !\"avoid\" U%s \"reach\" ]\n", strat, adv, bound.c_str());
      else
        o.print("P%s%s=? [ F%s \"reach\" ]\n", strat, adv, bound.c_str());
      if (!o.close()) return io_error(stem + ".pctl");
    }
    return IMDP_OK;
  });
}

}  // extern "C"
