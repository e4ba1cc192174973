// Test-only CPU twin of the paper's evaluation (Sec. 2 closed form, Eq. "fq",
// and the downward recursion, Eq. "r"), templated on the floating type so the
// same steps run in 24-bit (float), 53-bit (double), 64-bit (x86 long double)
// and 113-bit (__float128) arithmetic, as in the test program of Sec. 3.
// Q~ = q0 + q1 x + q2 x^2 u/v is evaluated either as root products (Eqs.
// "pz", "qz", "pqz") or from the expanded polynomial coefficients (Eq. "qr").
// This is neither the oracle nor the library: it exists to measure rounding
// errors of the method itself at several precisions.
//
// Input (text, one order per block, numbers as decimal strings):
//   n c q0 q1 q2 z K
//   <u root form> <v root form> <u expanded> <v expanded>
// where a root form is: P p_0 .. p_{P-1}  Q y_1 a_1 .. y_Q a_Q  L y_1 .. y_L
// (monic Horner part low -> high, quadratic factors (x - y)^2 + a, linear
// factors x - y) and an expanded polynomial is: E e_0 .. e_{E-1} (monic, low
// -> high).  The grid is x_i = float(z i / K), i = 0..K-1.
// Reference rows (long double, [K][n+1]) come from a binary file.
// Output, per precision and form: the max relative error of F_0, F_{n-1},
// F_n against the reference, and against the 113-bit root-form twin.
#include <quadmath.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

typedef __float128 quad;

template <class T> T parse(const char *s);
template <> float parse<float>(const char *s) { return strtof(s, nullptr); }
template <> double parse<double>(const char *s) { return strtod(s, nullptr); }
template <> long double parse<long double>(const char *s) { return strtold(s, nullptr); }
template <> quad parse<quad>(const char *s) { return strtoflt128(s, nullptr); }

inline float t_exp(float a) { return expf(a); }
inline double t_exp(double a) { return exp(a); }
inline long double t_exp(long double a) { return expl(a); }
inline quad t_exp(quad a) { return expq(a); }
inline float t_ldexp(float a, int e) { return ldexpf(a, e); }
inline double t_ldexp(double a, int e) { return ldexp(a, e); }
inline long double t_ldexp(long double a, int e) { return ldexpl(a, e); }
inline quad t_ldexp(quad a, int e) { return ldexpq(a, e); }
inline float t_frexp(float a, int *e) { return frexpf(a, e); }
inline double t_frexp(double a, int *e) { return frexp(a, e); }
inline long double t_frexp(long double a, int *e) { return frexpl(a, e); }
inline quad t_frexp(quad a, int *e) { return frexpq(a, e); }
inline float t_sqrt(float a) { return sqrtf(a); }
inline double t_sqrt(double a) { return sqrt(a); }
inline long double t_sqrt(long double a) { return sqrtl(a); }
inline quad t_sqrt(quad a) { return sqrtq(a); }

struct Text {
  std::vector<std::string> tok;
  size_t at = 0;
  const char *next() { return tok.at(at++).c_str(); }
  int next_int() { return atoi(next()); }
};

template <class T>
struct RootForm {
  std::vector<T> poly;                  // monic Horner part, low -> high
  std::vector<std::pair<T, T>> quadf;   // (x - y)^2 + a
  std::vector<T> lin;                   // x - y
  T eval(T x) const {
    T acc = T(1);
    if (poly.size() > 1) {
      T h = x + poly[poly.size() - 2];
      for (int k = (int)poly.size() - 3; k >= 0; --k) h = h * x + poly[k];
      acc = h;
    }
    for (auto &f : quadf) {
      const T t = x - f.first;
      acc = acc * (t * t + f.second);
    }
    for (auto &y : lin) acc = acc * (x - y);
    return acc;
  }
};

template <class T>
struct Expanded {
  std::vector<T> c;  // low -> high, monic
  T eval(T x) const {
    T acc = c.back();
    for (int k = (int)c.size() - 2; k >= 0; --k) acc = acc * x + c[k];
    return acc;
  }
};

struct Block {
  int n, K;
  std::vector<std::string> head;  // c q0 q1 q2 z
  std::vector<std::string> ur, vr, ue, ve;
};

template <class T>
RootForm<T> root_form(const std::vector<std::string> &s) {
  RootForm<T> r;
  size_t i = 0;
  int P = atoi(s[i++].c_str());
  for (int k = 0; k < P; ++k) r.poly.push_back(parse<T>(s[i++].c_str()));
  int Q = atoi(s[i++].c_str());
  for (int k = 0; k < Q; ++k) {
    T y = parse<T>(s[i++].c_str());
    T a = parse<T>(s[i++].c_str());
    r.quadf.push_back({y, a});
  }
  int L = atoi(s[i++].c_str());
  for (int k = 0; k < L; ++k) r.lin.push_back(parse<T>(s[i++].c_str()));
  return r;
}

template <class T>
Expanded<T> expanded(const std::vector<std::string> &s) {
  Expanded<T> e;
  int E = atoi(s[0].c_str());
  for (int k = 0; k < E; ++k) e.c.push_back(parse<T>(s[1 + k].c_str()));
  return e;
}

// v = m 4^j with m in [1/4, 1): sqrt(v) = sqrt(m) 2^j and v^k = m^k 4^(jk)
// exactly, so powers can be formed on m and rescaled once.  At n = 36 in
// single precision Q^n, D^n and c_n would leave the float range although
// Q^n sqrt(Q) e^{-x} and F_n do not; the split keeps every rounding the
// plain formula makes and only moves the exponent.
template <class T>
T split4(T v, int &j) {
  int e = 0;
  const T m = t_frexp(v, &e);  // v = m 2^e, m in [1/2, 1)
  j = (e + 1) >> 1;            // 2j >= e
  return t_ldexp(m, e - 2 * j);
}

// Q^n by repeated squaring (as the paper's unrolled code would)
template <class T>
T ipow(T a, int n) {
  T r = T(1);
  while (n) {
    if (n & 1) r = r * a;
    a = a * a;
    n >>= 1;
  }
  return r;
}

// F_0..F_n at x in type T: Eq. "fq" for F_n, then Eq. "r" downward (the
// printed denominator 2m+1 of F_{m-1} read as 2m-1), sharing e^{-x}.
// c_n is passed as cm 2^ce (cm in [1/2, 1)).
template <class T, class U, class V>
void row(const U &u, const V &v, T cm, int ce, T q0, T q1, T q2, int n, T x, T *F) {
  const T Q = q0 + q1 * x + q2 * x * x * (u.eval(x) / v.eval(x));
  int jq = 0, jd = 0, je = 0;
  const T Qm = split4(Q, jq);
  const T e = t_exp(-x);
  const T em = t_frexp(e, &je);  // e^{-x} near z_nb is below 2^-80: keep its exponent apart too
  const T D = x + t_ldexp(ipow(Qm, n) * t_sqrt(Qm) * em, jq * (2 * n + 1) + je);  // Q^s e^{-x}
  const T Dm = split4(D, jd);
  T f = t_ldexp(cm / (ipow(Dm, n) * t_sqrt(Dm)), ce - jd * (2 * n + 1));  // c_n D^{-s}
  F[n] = f;
  for (int m = n; m >= 1; --m) {
    f = (T(2) * x * f + e) / T(2 * m - 1);
    F[m - 1] = f;
  }
}

template <class T>
static double relerr(T got, long double ref) {
  if (ref == 0.0L) return 0.0;
  const long double d = (long double)got / ref - 1.0L;
  return (double)fabsl(d);
}

static double relq(quad got, quad ref) {
  if (ref == 0) return 0.0;
  return (double)fabsq(got / ref - 1);
}

template <class T>
void run(const char *name, const Block &b, const std::vector<long double> &ref, const std::vector<quad> &q) {
  const int n = b.n, K = b.K, W = n + 1;
  int ce = 0;  // c_n overflows a float from n = 35 on: split it in 113 bits, round the fraction
  const T cm = (T)t_frexp(parse<quad>(b.head[0].c_str()), &ce);
  const T q0 = parse<T>(b.head[1].c_str()), q1 = parse<T>(b.head[2].c_str()), q2 = parse<T>(b.head[3].c_str());
  const double z = strtod(b.head[4].c_str(), nullptr);
  const RootForm<T> ur = root_form<T>(b.ur), vr = root_form<T>(b.vr);
  const Expanded<T> ue = expanded<T>(b.ue), ve = expanded<T>(b.ve);
  for (int form = 0; form < 2; ++form) {
    double e_ref[3] = {0, 0, 0}, e_q[3] = {0, 0, 0};
    std::vector<T> F(W);
    for (int i = 0; i < K; ++i) {
      const float xf = (float)(z * i / K);
      const T x = (T)xf;
      if (form == 0) row<T>(ur, vr, cm, ce, q0, q1, q2, n, x, F.data());
      else row<T>(ue, ve, cm, ce, q0, q1, q2, n, x, F.data());
      const int ms[3] = {0, n > 0 ? n - 1 : 0, n};
      for (int k = 0; k < 3; ++k) {
        const int m = ms[k];
        const double a = relerr<T>(F[m], ref[(size_t)i * W + m]);
        const double r = relq((quad)F[m], q[(size_t)i * W + m]);
        if (a > e_ref[k]) e_ref[k] = a;
        if (r > e_q[k]) e_q[k] = r;
      }
    }
    printf("%s %s %d %.6e %.6e %.6e %.6e %.6e %.6e\n", name, form == 0 ? "root" : "expanded", n, e_ref[0], e_ref[1],
           e_ref[2], e_q[0], e_q[1], e_q[2]);
  }
}

int main(int argc, char **argv) {
  if (argc < 4) {
    fprintf(stderr, "usage: %s coeffs.txt refs.bin precision[,precision...]\n", argv[0]);
    return 2;
  }
  FILE *fh = fopen(argv[1], "r");
  if (!fh) return 3;
  std::vector<Block> blocks;
  char line[1 << 16];
  std::vector<std::vector<std::string>> lines;
  while (fgets(line, sizeof line, fh)) {
    std::vector<std::string> t;
    for (char *p = strtok(line, " \t\r\n"); p; p = strtok(nullptr, " \t\r\n")) t.push_back(p);
    if (!t.empty()) lines.push_back(t);
  }
  fclose(fh);
  for (size_t i = 0; i + 4 < lines.size(); i += 5) {
    Block b;
    b.n = atoi(lines[i][0].c_str());
    b.head.assign(lines[i].begin() + 1, lines[i].begin() + 6);
    b.K = atoi(lines[i][6].c_str());
    b.ur = lines[i + 1];
    b.vr = lines[i + 2];
    b.ue = lines[i + 3];
    b.ve = lines[i + 4];
    blocks.push_back(b);
  }
  FILE *rf = fopen(argv[2], "rb");
  if (!rf) return 4;
  const std::string prec = argv[3];
  for (const Block &b : blocks) {
    const size_t total = (size_t)b.K * (b.n + 1);
    std::vector<long double> ref(total);
    if (fread(ref.data(), sizeof(long double), total, rf) != total) return 5;
    // the 113-bit root-form rows: the rounding-free baseline of each order
    std::vector<quad> q(total);
    {
      int ce = 0;
      const quad cm = t_frexp(parse<quad>(b.head[0].c_str()), &ce);
      const quad q0 = parse<quad>(b.head[1].c_str()), q1 = parse<quad>(b.head[2].c_str()),
                 q2 = parse<quad>(b.head[3].c_str());
      const double z = strtod(b.head[4].c_str(), nullptr);
      const RootForm<quad> ur = root_form<quad>(b.ur), vr = root_form<quad>(b.vr);
      for (int i = 0; i < b.K; ++i) {
        const float xf = (float)(z * i / b.K);
        row<quad>(ur, vr, cm, ce, q0, q1, q2, b.n, (quad)xf, &q[(size_t)i * (b.n + 1)]);
      }
    }
    if (prec.find("24") != std::string::npos) run<float>("24", b, ref, q);
    if (prec.find("53") != std::string::npos) run<double>("53", b, ref, q);
    if (prec.find("64") != std::string::npos) run<long double>("64", b, ref, q);
    if (prec.find("113") != std::string::npos) run<quad>("113", b, ref, q);
  }
  return 0;
}
