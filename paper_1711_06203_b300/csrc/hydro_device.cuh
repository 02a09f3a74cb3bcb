// Device-side arithmetic of the CTU-PPM step (FP64, sm_103a).
//
// Each function is one stage of the unsplit PPM scheme named in the paper
// (Sec. 3.2): gamma-law EOS conversion, Colella-Woodward flattening and PPM
// reconstruction, reference-state characteristic tracing, HLLC Riemann flux,
// and the conservative transverse correction of CTU.  Operation order is
// fixed (the same order every time a quantity is formed) so that a build with
// contraction disabled reproduces the scheme's FP64 arithmetic exactly.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hydro {

constexpr int NG = 4;  // ghost zones per side: the stencil reaches 4 zones
// primitive fields stored per zone on the grown box
enum { QRHO = 0, QU = 1, QV = 2, QW = 3, QP = 4, QC = 5, QRC = 6, QCR = 7, QIC2 = 8, NQ = 9 };

constexpr double FLAT_OMEGA1 = 0.75, FLAT_OMEGA2 = 10.0, FLAT_EPS = 0.33;
constexpr double SIXTH = 1.0 / 6.0, TWOTHIRDS = 2.0 / 3.0, THIRD = 1.0 / 3.0;

struct StepConst {
  double gamma, gm1, gm1inv;  // gamma, gamma - 1, 1/(gamma - 1)
  double small_dens, small_pres;
  double grav[3];
  double dt, hdt;             // dt, dt/2
  double dtdx[3];             // dt/dx per axis
  int dim, flatten, has_grav;
  int einfeldt;   // HLLC outer speeds from Roe averages
  int flux_grav;  // gravity energy source from the face mass fluxes
};

// ---------------------------------------------------------------- comparisons
// B300's FP64 pipe runs a compare (DSETP) or min/max at the same ~1.6
// lanes/clock/SM as an FMA, so every comparison of doubles here is done on
// the integer pipe from the bit pattern.  For finite (and infinite) values
// these reproduce IEEE comparison exactly, including +0 == -0.
// The compares themselves are inline PTX on 64-bit integers, so that the
// compiler cannot fold a bit-pattern compare back into an FP64 compare.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// signed 64-bit a < b, evaluated on the integer pipe
__device__ __forceinline__ bool ilt(long long a, long long b) {
  int r;
  asm("{\n\t.reg .pred p;\n\tsetp.lt.s64 p, %1, %2;\n\tselp.s32 %0, 1, 0, p;\n\t}" : "=r"(r) : "l"(a), "l"(b));
  return r != 0;
}
// The sign bit and the magnitude of a double's bit pattern, masked in inline
// PTX: the same masks written in C are recognised by the compiler as an FP64
// absolute value, negation or sign copy and then cost an FP64 instruction
// (measured: one FP64 add per mask when the operand comes from an FP64 op).
__device__ __forceinline__ long long sign_bits(double x) {
  long long r;
  asm("and.b64 %0, %1, 0x8000000000000000;" : "=l"(r) : "l"(dbits(x)));
  return r;
}
__device__ __forceinline__ long long mag_bits(double x) {
  long long r;
  asm("and.b64 %0, %1, 0x7FFFFFFFFFFFFFFF;" : "=l"(r) : "l"(dbits(x)));
  return r;
}
// x > 0: positive sign and nonzero magnitude
__device__ __forceinline__ bool gt0(double x) { return ilt(0, dbits(x)); }
// x < 0 <=> -x > 0
__device__ __forceinline__ bool lt0(double x) { return ilt(0, dbits(x) ^ (long long)0x8000000000000000ULL); }
__device__ __forceinline__ bool ge0(double x) { return !lt0(x); }
// order key: monotone in x, equal for +0 and -0
__device__ __forceinline__ long long okey(double x) {
  const long long m = mag_bits(x);
  return ilt(dbits(x), 0) ? -m : m;
}
__device__ __forceinline__ bool dless(double a, double b) { return ilt(okey(a), okey(b)); }
// min/max as explicit selects: ties return the first argument
__device__ __forceinline__ double dmin(double a, double b) { return dless(b, a) ? b : a; }
__device__ __forceinline__ double dmax(double a, double b) { return dless(a, b) ? b : a; }
// |x| by clearing the sign bit on the integer pipe (an FP64 absolute value
// whose only consumers are bit-pattern compares would otherwise cost an
// FP64 issue slot)
__device__ __forceinline__ double dabs(double x) { return __longlong_as_double(mag_bits(x)); }
// 2x and x/2 on the integer pipe, bitwise equal to the IEEE products 2.0 * x
// and 0.5 * x (round to nearest even) for every input: scaling by two moves
// the exponent field, except where the value is or becomes subnormal (the
// significand shifts, rounding half to even) or overflows.  An FP64 multiply
// costs an issue slot on the scarce FP64 pipe; these cost a few integer ops.
__device__ __forceinline__ double dtwice(double x) {
  const long long b = dbits(x);
  const long long sign = sign_bits(x), mag = mag_bits(x);
  const long long e = mag >> 52;
  long long r;
  if (e == 0) r = sign | (mag << 1);                        // zero or subnormal
  else if (e < 2046) r = b + (1LL << 52);                   // normal: exponent + 1
  else if (e == 2046) r = sign | 0x7FF0000000000000LL;      // overflow to infinity
  else r = b;                                               // infinity, NaN
  return __longlong_as_double(r);
}
__device__ __forceinline__ double dhalf(double x) {
  const long long b = dbits(x);
  const long long sign = sign_bits(x), mag = mag_bits(x);
  const long long e = mag >> 52;
  long long r;
  if (e >= 2 && e < 2047) {
    r = b - (1LL << 52);                                    // the half is normal
  } else if (e == 2047) {
    r = b;                                                  // infinity, NaN
  } else {
    // the half is subnormal: significand M (implicit bit included when
    // e == 1) halved, a dropped 1 rounding the quotient to even
    const long long q = mag >> 1;
    r = sign | (q + (mag & q & 1));
  }
  return __longlong_as_double(r);
}
// -x by flipping the sign bit on the integer pipe (a negated operand that
// feeds the integer-pipe product below would otherwise be formed on the FP64
// pipe; inline PTX for the reason given at sign_bits)
__device__ __forceinline__ double dneg(double x) {
  long long r;
  asm("xor.b64 %0, %1, 0x8000000000000000;" : "=l"(r) : "l"(dbits(x)));
  return __longlong_as_double(r);
}
// ---------------------------------------------------------------- FP64 products and sums on the integer pipe
// B300 issues FP64 arithmetic at 2 lanes per clock per SM, while each SM
// partition's integer ALU and IMAD pipes take 16 lanes per clock each.  A
// binary64 product rounded to nearest even, formed from the bit patterns
// (significand product in 32-bit limbs, normalise, round, repack), costs
// about 30 ALU and 15 IMAD instructions: roughly one native multiply's worth
// of issue time, but on other units.  Moving a share of a kernel's products
// (and, at about twice that cost, a few sums) there runs them beside the
// FP64 pipe instead of queueing on it.  Both functions return the IEEE
// result bit for bit (a GPU test compares them with the hardware operations
// over edge cases and random bit patterns), so the contraction-free build
// still performs exactly the oracle's operations.
// 32-bit unsigned a < b and a != b on the integer pipe
__device__ __forceinline__ bool ult32(unsigned a, unsigned b) {
  int r;
  asm("{\n\t.reg .pred p;\n\tsetp.lo.u32 p, %1, %2;\n\tselp.s32 %0, 1, 0, p;\n\t}" : "=r"(r) : "r"(a), "r"(b));
  return r != 0;
}
__device__ __forceinline__ bool ne32(unsigned a, unsigned b) {
  int r;
  asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, %2;\n\tselp.s32 %0, 1, 0, p;\n\t}" : "=r"(r) : "r"(a), "r"(b));
  return r != 0;
}
// a * b, IEEE binary64, round to nearest even.  Normal operands with a normal
// result, and zero operands, stay on the integer pipe; subnormal, infinite or
// NaN operands and results that over- or underflow take the FP64 multiply.
__device__ __forceinline__ double mul_i(double a, double b) {
  const unsigned long long ua = (unsigned long long)dbits(a), ub = (unsigned long long)dbits(b);
  const unsigned ah0 = (unsigned)(ua >> 32), bh0 = (unsigned)(ub >> 32), al = (unsigned)ua, bl = (unsigned)ub;
  const unsigned ea = (ah0 >> 20) & 0x7FFu, eb = (bh0 >> 20) & 0x7FFu;
  const unsigned ah = (ah0 & 0xFFFFFu) | 0x100000u, bh = (bh0 & 0xFFFFFu) | 0x100000u;
  // significands (ah:al)(bh:bl) = P = v 2^64 + w1 2^32 + w0, 2^104 <= P < 2^106
  const unsigned long long t = (unsigned long long)al * bl;
  const unsigned long long u = (unsigned long long)ah * bl + (t >> 32);
  const unsigned long long u2 = (unsigned long long)al * bh + u;
  const unsigned long long v = (unsigned long long)ah * bh + (u2 >> 32);
  const unsigned w1 = (unsigned)u2, w0 = (unsigned)t;
  const unsigned top = (unsigned)(v >> 41);  // P >= 2^105
  // 53-bit significand q = P >> (52 + top); guard bit below it; sticky below that
  unsigned long long q = (v << (12 - top)) | (unsigned long long)(w1 >> (20 + top));
  const unsigned guard = (w1 >> (19 + top)) & 1u;
  const unsigned sticky = (w1 & ((1u << (19 + top)) - 1u)) | w0;
  q += (unsigned long long)(guard & ((ne32(sticky, 0u) ? 1u : 0u) | ((unsigned)q & 1u)));
  const int e = (int)(ea + eb) - 1023 + (int)top;
  const unsigned long long sign = (unsigned long long)((ah0 ^ bh0) & 0x80000000u) << 32;
  // the significand's leading bit adds one to the exponent field, and a
  // rounding carry out of the significand adds one more
  unsigned long long r = ((((unsigned long long)(unsigned)(e - 1)) << 52) + q) | sign;
  const bool a_zero = !ne32((ah0 & 0x7FFFFFFFu) | al, 0u), b_zero = !ne32((bh0 & 0x7FFFFFFFu) | bl, 0u);
  const bool zero = (a_zero && ne32(eb, 0x7FFu)) || (b_zero && ne32(ea, 0x7FFu));
  const bool fast = ult32(ea - 1u, 2046u) && ult32(eb - 1u, 2046u) && ult32((unsigned)(e - 1), 2046u);
  if (__builtin_expect(!(fast || zero), 0)) r = (unsigned long long)dbits(__dmul_rn(a, b));
  r = zero ? sign : r;
  return __longlong_as_double((long long)r);
}
// a + b, IEEE binary64, round to nearest even, for every input (an invalid
// operation returns a NaN).
__device__ __forceinline__ double add_i(double a, double b) {
  const unsigned long long FRAC = 0x000FFFFFFFFFFFFFull, IMPL = 1ull << 52;
  const unsigned long long ua = (unsigned long long)dbits(a), ub = (unsigned long long)dbits(b);
  const unsigned long long aa = (unsigned long long)mag_bits(a), ab = (unsigned long long)mag_bits(b);
  // order by magnitude (the sign of the difference of two values < 2^63)
  const bool swap = (long long)(aa - ab) < 0;
  const unsigned long long x = swap ? ub : ua, y = swap ? ua : ub;
  const unsigned long long xm = swap ? ab : aa, ym = swap ? aa : ab;
  const unsigned long long xsign = (unsigned long long)((unsigned)(x >> 32) & 0x80000000u) << 32;
  const unsigned xh = (unsigned)(xm >> 32), yh = (unsigned)(ym >> 32);
  int ex = (int)(xh >> 20), ey = (int)(yh >> 20);
  // significands with 10 guard bits; a subnormal has exponent 1 and no leading bit
  unsigned long long mx = ((xm & FRAC) | (ne32((unsigned)ex, 0u) ? IMPL : 0ull)) << 10;
  unsigned long long my = ((ym & FRAC) | (ne32((unsigned)ey, 0u) ? IMPL : 0ull)) << 10;
  ex = max(ex, 1);
  ey = max(ey, 1);
  const int d = min(ex - ey, 63);
  const unsigned long long lost = my << (64 - d);  // the bits the alignment drops (none for d = 0)
  my = (my >> d) | (ne32((unsigned)(lost >> 32) | (unsigned)lost, 0u) ? 1ull : 0ull);
  const bool sub = (int)((unsigned)(x >> 32) ^ (unsigned)(y >> 32)) < 0;
  unsigned long long s = mx + (sub ? (0ull - my) : my);
  const int carry = (int)(s >> 63);
  s = carry ? ((s >> 1) | (s & 1ull)) : s;
  int e = ex + carry;
  const unsigned sh_hi = (unsigned)(s >> 32), sh_lo = (unsigned)s;
  const bool nonzero = ne32(sh_hi | sh_lo, 0u);
  const int lz = (ne32(sh_hi, 0u) ? __clz(sh_hi) : 32 + __clz(sh_lo)) - 1;
  const int sh = min(lz, e - 1);  // normalise, but not below the smallest exponent
  s <<= sh;
  e -= sh;
  const unsigned long long q = (s + 0x1FFull + ((s >> 10) & 1ull)) >> 10;  // round half to even
  unsigned long long r = ((unsigned long long)(e - 1) << 52) + q;
  r = ult32((unsigned)(r >> 32), 0x7FF00000u) ? r : 0x7FF0000000000000ull;  // overflow
  r |= xsign;
  r = nonzero ? r : (sub ? 0ull : xsign);  // exact zero: +0 unless both -0
  // an infinite or NaN operand is the one of larger magnitude
  const bool special = !ult32(xh, 0x7FF00000u);
  const bool nan = ne32((xh & 0xFFFFFu) | (unsigned)xm, 0u) || (!ult32(yh, 0x7FF00000u) && sub);
  r = special ? (nan ? 0x7FFFFFFFFFFFFFFFull : x) : r;
  return __longlong_as_double((long long)r);
}// Reciprocal, quotient and square root.  The contraction-free build keeps the
// IEEE operations, so it agrees with the oracle bit for bit.  The product
// build refines the hardware's approximate reciprocal and reciprocal square
// root on the FMA pipe: one third-order step r' = r + r (e + e^2), e = 1 - x r,
// for 1/x; y' = y + y (1 - x y^2)/2 once, then s = x y corrected by
// s + (x - s^2) y/2 for sqrt(x).  On the FP64 pipe that is 3 (1/x and a/b,
// whose final product runs on the integer pipe) and 4 (sqrt) fused
// multiply-adds, against about 5.7, 8.6 and 8.6 issue slots measured for the
// IEEE operations; the results stay within 2 ulp (a GPU test bounds the error).
// Arguments outside [2^-959, 2^960], zero, negative or non-finite take the
// IEEE path.  Both refinements are the truncated-series (higher-order
// Newton-Raphson) corrections of an approximate reciprocal and reciprocal
// square root, as described for FMA hardware in J.-M. Muller et al.,
// "Handbook of Floating-Point Arithmetic", 2nd ed. (Birkhaeuser, 2018), in its
// treatment of division and square root by Newton-Raphson iterations.
#ifdef HYDRO_IEEE_DIV_SQRT
__device__ __forceinline__ double drcp(double x) { return 1.0 / x; }
__device__ __forceinline__ double ddiv(double a, double b) { return a / b; }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
#else
// positive and normal with exponent field in [64, 1983]
__device__ __forceinline__ bool newton_range(double x) {
  return (unsigned long long)((dbits(x) >> 52) - 64) < 1920ull;
}
__device__ __forceinline__ double rcp_newton(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  // one third-order step: with r = (1 - e)/x, r (1 + e + e^2) = (1 - e^3)/x
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double drcp(double x) {
  const double ax = dabs(x);
  if (__builtin_expect(!newton_range(ax), 0)) return 1.0 / x;
  const double r = rcp_newton(ax);
  return __longlong_as_double(dbits(r) | sign_bits(x));
}
__device__ __forceinline__ double ddiv(double a, double b) {
  const double ab = dabs(b);
  if (__builtin_expect(!newton_range(ab), 0)) return a / b;
  const double r = rcp_newton(ab);
  return mul_i(a, __longlong_as_double(dbits(r) | sign_bits(b)));
}
// 1/sqrt(x) for x in the refined range: from the hardware estimate y with
// e = 1 - x y^2, 1/sqrt(x) = y (1 - e)^(-1/2) = y (1 + e/2 + 3e^2/8 + ...),
// the binomial series kept to second order (error 5e^3/16)
__device__ __forceinline__ double rsqrt_newton(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-mul_i(x, y), y, 1.0);
  return fma(y, e * fma(0.375, e, 0.5), y);
}
__device__ __forceinline__ double dsqrt(double x) {
  if (__builtin_expect(!newton_range(x), 0)) return sqrt(x);
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-mul_i(x, y), y, 1.0);
  y = fma(dhalf(e), y, y);
  const double sq = mul_i(x, y);
  return fma(fma(-sq, sq, x), dhalf(y), sq);
}
#endif
// operands known to be >= +0 (magnitudes, pressures, speeds): raw bits order
__device__ __forceinline__ double dmin_nn(double a, double b) { return ilt(dbits(b), dbits(a)) ? b : a; }
__device__ __forceinline__ double dmax_nn(double a, double b) { return ilt(dbits(a), dbits(b)) ? b : a; }
// |x| > y for y >= +0
__device__ __forceinline__ bool abs_gt(double x, double y) {
  return ilt(dbits(y), mag_bits(x));
}
// signed 64-bit a != b on the integer pipe (a bit-pattern "x != 0" written in
// C would be recognised as the FP64 compare x != 0.0)
__device__ __forceinline__ bool ine(long long a, long long b) {
  int r;
  asm("{\n\t.reg .pred p;\n\tsetp.ne.s64 p, %1, %2;\n\tselp.s32 %0, 1, 0, p;\n\t}" : "=r"(r) : "l"(a), "l"(b));
  return r != 0;
}
// x + (+0.0) as an integer select: x itself, except that -0 becomes +0
__device__ __forceinline__ double pz(double x) {
  const long long b = dbits(x);
  return __longlong_as_double(ine(b, (long long)0x8000000000000000ULL) ? b : 0LL);
}
// a and b nonzero with the same sign
__device__ __forceinline__ bool same_sign_strict(double a, double b) {
  long long ba = dbits(a), bb = dbits(b);
  bool nz = ine(ba << 1, 0) & ine(bb << 1, 0);
  return nz & !ilt(ba ^ bb, 0);
}
// finite: exponent field not all ones
__device__ __forceinline__ bool dfinite(double x) { return ine((dbits(x) >> 52) & 0x7FF, 0x7FF); }

// ---------------------------------------------------------------- EOS
// conserved -> primitive with floors; sets *bad for a non-physical state
__device__ __forceinline__ void cons_to_prim_flag(const double U[5], const StepConst& K, double q[5],
                                                  double* inv_out, bool* bad) {
  double rho = U[0];
  if (!(gt0(rho) && dfinite(rho))) *bad = true;
  rho = dmax(rho, K.small_dens);
  double inv = drcp(rho);
  double u = mul_i(U[1], inv), v = mul_i(U[2], inv), w = mul_i(U[3], inv);
  double ke = dhalf(rho) * ((mul_i(u, u) + v * v) + w * w);
  double p = mul_i(K.gm1, U[4] - ke);
  if (!(gt0(p) && dfinite(p) && dfinite(U[1]) && dfinite(U[2]) && dfinite(U[3]))) *bad = true;
  p = dmax(p, K.small_pres);
  q[0] = rho; q[1] = u; q[2] = v; q[3] = w; q[4] = p;
  *inv_out = inv;
}

// face state for the Riemann solver: rho, u, v, w, p, rho*E, 1/rho
enum { S_RHO = 0, S_P = 4, S_E = 5, S_INV = 6, NS = 7 };

// sound speed sqrt(gamma p / rho) of a face state
__device__ __forceinline__ double sound_of(const double s[NS], const StepConst& K) {
  return dsqrt(mul_i(mul_i(K.gamma, s[S_P]), s[S_INV]));
}

__device__ __forceinline__ double energy_of(const double q[5], const StepConst& K) {
  return q[4] * K.gm1inv + mul_i(dhalf(q[0]), (mul_i(q[1], q[1]) + q[2] * q[2]) + q[3] * q[3]);
}

__device__ __forceinline__ void state_from_prim(const double q[5], const StepConst& K, double s[NS]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) s[c] = q[c];
  s[S_E] = energy_of(q, K);
  s[S_INV] = drcp(q[0]);
}

// the same with the state's sound speed: in the product build 1/rho and
// sqrt(gamma p / rho) both come from one refined y = 1/sqrt(gamma p rho),
// as c = (gamma p) y and 1/rho = c y, instead of a reciprocal and a square root
__device__ __forceinline__ void state_from_prim_c(const double q[5], const StepConst& K, double s[NS], double* c) {
#pragma unroll
  for (int v = 0; v < 5; ++v) s[v] = q[v];
  s[S_E] = energy_of(q, K);
#ifndef HYDRO_IEEE_DIV_SQRT
  // (the three products after gamma p run on the FP64 pipe: measured 7 %
  // faster in the first solves than on the integer pipe, which there already
  // carries the sign tests and the other moved products, 60 % busy)
  const double gp = mul_i(K.gamma, q[4]);
  const double x = gp * q[0];
  if (__builtin_expect(newton_range(x), 1)) {
    const double y = rsqrt_newton(x);
    *c = gp * y;
    s[S_INV] = *c * y;
    return;
  }
#endif
  s[S_INV] = drcp(q[0]);
  *c = sound_of(s, K);
}

__device__ __forceinline__ void state_from_cons(const double U[5], const StepConst& K, double s[NS]) {
  double rho = dmax(U[0], K.small_dens);
  double inv = drcp(rho);
  double u = mul_i(U[1], inv), v = mul_i(U[2], inv), w = mul_i(U[3], inv);
  double ke = dhalf(rho) * ((mul_i(u, u) + v * v) + w * w);
  double p = mul_i(K.gm1, U[4] - ke);
  p = dmax(p, K.small_pres);
  s[0] = rho; s[1] = u; s[2] = v; s[3] = w; s[4] = p;
  s[S_E] = U[4];
  s[S_INV] = inv;
}

// ---------------------------------------------------------------- flattening (CW84 App. A)
// chi~ of zone j from p_{j-2..j+2} and the normal velocities u_{j-1}, u_{j+1}
__device__ __forceinline__ double flat_tilde(double pm2, double pm1, double pp1, double pp2, double um1, double up1,
                                             double small_pres) {
  double dp1 = pp1 - pm1;
  double dp2 = pp2 - pm2;
  // u_{j-1} - u_{j+1} > 0 as an order comparison (a rounded difference has
  // the sign of the exact one and vanishes only for equal operands)
  if (dless(up1, um1) && abs_gt(dp1, mul_i(FLAT_EPS, dmin_nn(pp1, pm1)))) {
    double z = dabs(dp1) / dmax_nn(dabs(dp2), small_pres);
    double f = dmax(0.0, dmin(1.0, mul_i(FLAT_OMEGA2, z - FLAT_OMEGA1)));
    return 1.0 - f;
  }
  return 1.0;
}

// ---------------------------------------------------------------- PPM (CW84 eqs. 1.6-1.10)
// monotonised centred slope of the middle zone of (am1, a0, ap1), given its
// one-sided differences dl = a0 - am1 and dr = ap1 - a0 (a pencil sweep
// forms each difference once: one zone's dr is the next zone's dl)
__device__ __forceinline__ double mc_slope_d(double dl, double dr, double am1, double ap1) {
  if (!same_sign_strict(dl, dr)) return 0.0;
  double da = dhalf(ap1 - am1);
  // 2 min(|dl|, |dr|) == min(2|dl|, 2|dr|) exactly (doubling is exact)
  double m2 = dtwice(dmin_nn(dabs(dl), dabs(dr)));
  double lim = dmin_nn(dabs(da), m2);
  return __longlong_as_double(dbits(lim) | sign_bits(da));  // lim >= 0: copy the sign of da
}
__device__ __forceinline__ double mc_slope(double am1, double a0, double ap1) {
  return mc_slope_d(a0 - am1, ap1 - a0, am1, ap1);
}

// interface value between zones with averages a0, a1 and slopes s0, s1
__device__ __forceinline__ double face_value(double a0, double a1, double s0, double s1) {
  return dhalf(a0 + a1) - SIXTH * (s1 - s0);
}

// limited, flattened parabola of a zone: average ai, interface values aM, aP
// The scheme's sign tests on differences -- (aP - ai)(ai - aM) > 0 and the
// signs of M - D/6 and M + D/6 -- are taken as order comparisons of the
// operands: a rounded difference has the sign of the exact one and is zero
// only when the operands are equal, so every decision is the one the
// differences would give, without forming them on the FP64 pipe.
// (dap, optional, receives ap - am, formed once here: the limiter's D when the
// edges were left unchanged)
__device__ __forceinline__ void ppm_limit(double ai, double aM, double aP, double chi, double& am, double& ap,
                                          double& a6, double* dap = nullptr) {
  const long long ki = okey(ai), kP = okey(aP), kM = okey(aM);
  double M = 0.0;  // ai - (aM + aP)/2 for the current edges
  double dd = 0.0;  // aP - aM for the current edges
  bool m_current = true;
  if (!((ilt(ki, kP) && ilt(kM, ki)) || (ilt(kP, ki) && ilt(ki, kM)))) {
    aP = ai; aM = ai;  // a local extremum: flat, and ai - (ai + ai)/2 = +0
  } else {
    const double D = aP - aM;
    dd = D;
    M = ai - dhalf(aM + aP);
    const long long kD = okey(D), km = okey(M), kt = okey(SIXTH * D);  // t = D/6
    // up = M - t, dn = M + t; D != 0 here.  Either edge may be reset from
    // the other (a- = 3 ai - 2 a+, else a+ = 3 ai - 2 a-): one operation on
    // the selected edge, so lanes taking different cases share it
    const bool dpos = ilt(0, kD);
    const bool set_m = dpos ? ilt(kt, km) : ilt(km, kt);
    const bool set_p = !set_m && (dpos ? ilt(km, -kt) : ilt(-kt, km));
    if (set_m || set_p) {
      const double y = 3.0 * ai - dtwice(set_m ? aP : aM);
      aM = set_m ? y : aM;
      aP = set_p ? y : aP;
      m_current = false;
    }
  }
  if (ilt(dbits(chi), dbits(1.0))) {  // chi < 1 (chi is in [0, 1]): blend toward the average
    aP = mul_i(chi, aP) + (1.0 - chi) * ai;
    aM = mul_i(chi, aM) + (1.0 - chi) * ai;
    m_current = false;
  }
  if (!m_current) {
    M = ai - dhalf(aM + aP);
    dd = aP - aM;
  }
  if (dap) *dap = dd;
  am = aM; ap = aP; a6 = 6.0 * M;
}

// averages of the parabola over the part of the zone swept by a wave of
// Courant number s toward the high (I+) / low (I-) face
// dap = ap - am
__device__ __forceinline__ double integ_plus(double am, double ap, double dap, double a6, double s) {
  return ap - dhalf(s) * (dap - (1.0 - TWOTHIRDS * s) * a6);
}
__device__ __forceinline__ double integ_minus(double am, double ap, double dap, double a6, double s) {
  return am + dhalf(s) * (dap + (1.0 - TWOTHIRDS * s) * a6);
}

// ---------------------------------------------------------------- HLLC (Toro-Spruce-Speares)
// returns true when the flux is taken from the left side of the fan (S* >= 0).
// Outer wave speeds: Einfeldt's (EINF) or Davis's, fixed at compile time; the
// solver kernels are instantiated for each and chosen at launch from
// K.einfeldt, so a Davis kernel carries none of the Einfeldt code and its
// registers (compiled together they raised every solver kernel's
// allocation from 64 to 76-96 registers).
// HLLC flux of two face states whose sound speeds cl, cr are given
template <bool EINF>
__device__ __forceinline__ bool hllc_flux_c(const double sL[NS], const double sR[NS], double cl, double cr, int d,
                                            const StepConst& K, double F[5]) {
  double rl = sL[S_RHO], pl = sL[S_P], ul = sL[1 + d];
  double rr = sR[S_RHO], pr = sR[S_P], ur = sR[1 + d];
  double sl, sr;
  if (!EINF) {  // Davis
    sl = dmin(ul - cl, ur - cr);
    sr = dmax(ul + cl, ur + cr);
  } else {  // Einfeldt: Roe-averaged normal velocity and sound speed
#ifdef HYDRO_IEEE_DIV_SQRT
    double ql = dsqrt(rl), qr = dsqrt(rr);
    double iw = drcp(ql + qr);
    double wl = mul_i(ql, iw), wr = mul_i(qr, iw);
#else
    // the Roe weights sqrt(rl)/(sqrt(rl) + sqrt(rr)) = 1/(1 + sqrt(rr/rl))
    // and 1 minus it: one square root and one reciprocal instead of two and one
    const double wl = drcp(1.0 + dsqrt(mul_i(rr, sL[S_INV]))), wr = 1.0 - wl;
#endif
    double ut0 = wl * sL[1] + mul_i(wr, sR[1]), ut1 = wl * sL[2] + mul_i(wr, sR[2]);
    double ut2 = wl * sL[3] + mul_i(wr, sR[3]);
    double hl = mul_i(sL[S_E] + pl, sL[S_INV]), hr = mul_i(sR[S_E] + pr, sR[S_INV]);
    double ht = wl * hl + mul_i(wr, hr);
    double q2 = (mul_i(ut0, ut0) + ut1 * ut1) + ut2 * ut2;
    double ct = dsqrt(mul_i(K.gm1, ht - dhalf(q2)));
    double utn = (d == 0) ? ut0 : (d == 1) ? ut1 : ut2;
    sl = dmin(ul - cl, utn - ct);
    sr = dmax(ur + cr, utn + ct);
  }
  double ml = mul_i(rl, sl - ul), mr = mul_i(rr, sr - ur);
  const double num = (pr - pl) + ml * ul - mr * ur, den = ml - mr;
#ifdef HYDRO_IEEE_DIV_SQRT
  const double sstar = ddiv(num, den);
  const bool sstar_ge0 = ge0(sstar);
#else
  // the sign of S* = num/den without forming the quotient: a zero numerator
  // gives +-0 (>= 0), otherwise the quotient is >= 0 when the signs agree
  const bool sstar_ge0 = !ine(dbits(num) << 1, 0) || !ilt(dbits(num) ^ dbits(den), 0);
#endif
  int region = ge0(sl) ? 0 : sstar_ge0 ? 1 : gt0(sr) ? 2 : 3;
  bool left = region <= 1;
  // the chosen side's state, component by component (selecting a pointer to
  // one of the two arrays would force both into local memory)
  double s[NS];
#pragma unroll
  for (int c = 0; c < NS; ++c) s[c] = left ? sL[c] : sR[c];
  double rho = s[S_RHO], un = s[1 + d], p = s[S_P], E = s[S_E];
  if (region == 0 || region == 3) {
    // physical flux of the chosen side
    double mass = mul_i(rho, un);
    F[0] = mass;
#pragma unroll
    for (int k = 0; k < 3; ++k) F[1 + k] = (k == d) ? mass * un + p : mul_i(mass, s[1 + k]);
    F[4] = mul_i(un, E + p);
    return left;
  }
  // star region: F_K + S_K (U*_K - U_K) evaluated as the physical flux of the
  // star state, with f = rho (S_K - u)/(S_K - S*), p* = p + rho (S_K - u)(S* - u)
  // and (rho E)* = f E/rho + (S* - u)(f S* + p/(S_K - S*))
  double sk = left ? sl : sr, mk = left ? ml : mr;
#ifdef HYDRO_IEEE_DIV_SQRT
  double r = drcp(sk - sstar);
#else
  // S* = num/den and r = 1/(S_K - S*) = den/q with q = S_K den - num, both
  // from one reciprocal g = 1/(den q): 1/den = g q, 1/q = g den
  const double q = fma(sk, den, -num);
  const double g = drcp(mul_i(den, q));
  const double sstar = mul_i(num, mul_i(g, q));
  const double r = mul_i(den, mul_i(g, den));
#endif
  double f = mul_i(mk, r);
  double du = sstar - un;
  double mstar = mul_i(f, sstar);
  double pstar = p + mk * du;
  double Estar = f * mul_i(E, s[S_INV]) + mul_i(du, mstar + p * r);
  F[0] = mstar;
#pragma unroll
  for (int k = 0; k < 3; ++k) F[1 + k] = (k == d) ? mstar * sstar + pstar : mul_i(mstar, s[1 + k]);
  F[4] = mul_i(sstar, Estar + pstar);
  return left;
}

template <bool EINF>
__device__ __forceinline__ bool hllc_flux(const double sL[NS], const double sR[NS], int d, const StepConst& K,
                                          double F[5]) {
  return hllc_flux_c<EINF>(sL, sR, sound_of(sL, K), sound_of(sR, K), d, K, F);
}

}  // namespace hydro
