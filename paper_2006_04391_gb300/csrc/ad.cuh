// Expression-template automatic differentiation held in registers.
//
// AutoMat (arXiv 2006.04391) Sec. 5 evaluates the partials of the two
// potentials with the reverse mode of AD on the expression level: a scalar
// expression is turned into a tree of node objects by operator overloading;
// a forward sweep evaluates it, a reverse sweep propagates adjoints to the
// leaves with the chain rule (Fig. "reverse_mode").  Second derivatives come
// from explicit second-order types, and passive ("lower order") arguments do
// not receive adjoints.
//
// Design here (sm_103a, one CUDA thread per voxel, every node in registers):
//  * Nodes cache their forward value (the "tape" is the set of node objects,
//    all of them scalar-replaced into registers after inlining).  On GB300 the
//    FP64 pipe is the bottleneck (about 1/61 of FP32), so re-evaluating a
//    sub-expression in the reverse sweep -- the paper's choice to save
//    registers on Volta -- would cost FP64 issue slots; registers are cheap.
//  * Second order is forward-over-reverse: the reverse sweep runs on Tan
//    numbers (value + N tangent components), so the adjoint of leaf k comes
//    out as (df/dx_k, sum_j d2f/dx_k dx_j t_j).  Seeding the leaves with unit
//    tangents gives gradient and Hessian in one sweep (vector mode), seeding
//    with a direction gives a Hessian-vector product.
//  * The tangent sparsity is a template parameter (bit mask M): operations on
//    components that are structurally zero are removed at compile time.  IEEE
//    arithmetic forbids the compiler to fold 0*x, so without the masks a
//    quadratic potential would pay runtime FP64 work for constant Hessians.
//  * Passive leaves (Cst) take no adjoint (the paper's mixed-order nodes).
//  * Leaf adjoint accumulators start at -0.0, the additive identity that the
//    compiler may fold (-0.0 + x == x for every x).
//
// The header compiles for the host as well (g++), which the CPU tests use to
// check it against finite differences.
#pragma once

#include <cmath>
#include <type_traits>
#include <utility>

#if defined(__CUDACC__)
#define AD_HD __host__ __device__ __forceinline__
#else
#define AD_HD inline
#endif

#include "fpow.cuh"

namespace gsm {
namespace ad {

// ------------------------------------------------------------------ numbers

template <class T, int N, unsigned M>
struct Tan {
  T v;
  T d[N];
  static constexpr unsigned mask = M;
};

template <class X> struct tan_info { static constexpr bool is_tan = false; };
template <class T, int N, unsigned M> struct tan_info<Tan<T, N, M>> {
  static constexpr bool is_tan = true;
  static constexpr int n = N;
  static constexpr unsigned mask = M;
  using scalar = T;
};

template <class X> struct scalar_of { using type = X; };
template <class T, int N, unsigned M> struct scalar_of<Tan<T, N, M>> { using type = T; };
template <class X> using scalar_of_t = typename scalar_of<X>::type;

template <unsigned M> AD_HD constexpr bool has(int k) { return ((M >> k) & 1u) != 0u; }

template <class T> AD_HD T value_of(const T& x) { return x; }
template <class T, int N, unsigned M> AD_HD T value_of(const Tan<T, N, M>& x) { return x.v; }

// Tan (op) Tan -----------------------------------------------------------------
template <class T, int N, unsigned A, unsigned B>
AD_HD Tan<T, N, A | B> operator+(const Tan<T, N, A>& x, const Tan<T, N, B>& y) {
  Tan<T, N, A | B> r;
  r.v = x.v + y.v;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (has<A>(k) && has<B>(k)) r.d[k] = x.d[k] + y.d[k];
    else if (has<A>(k)) r.d[k] = x.d[k];
    else if (has<B>(k)) r.d[k] = y.d[k];
    else r.d[k] = T(0);
  }
  return r;
}

template <class T, int N, unsigned A, unsigned B>
AD_HD Tan<T, N, A | B> operator-(const Tan<T, N, A>& x, const Tan<T, N, B>& y) {
  Tan<T, N, A | B> r;
  r.v = x.v - y.v;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (has<A>(k) && has<B>(k)) r.d[k] = x.d[k] - y.d[k];
    else if (has<A>(k)) r.d[k] = x.d[k];
    else if (has<B>(k)) r.d[k] = -y.d[k];
    else r.d[k] = T(0);
  }
  return r;
}

template <class T, int N, unsigned A, unsigned B>
AD_HD Tan<T, N, A | B> operator*(const Tan<T, N, A>& x, const Tan<T, N, B>& y) {
  Tan<T, N, A | B> r;
  r.v = x.v * y.v;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (has<A>(k) && has<B>(k)) r.d[k] = x.d[k] * y.v + x.v * y.d[k];
    else if (has<A>(k)) r.d[k] = x.d[k] * y.v;
    else if (has<B>(k)) r.d[k] = x.v * y.d[k];
    else r.d[k] = T(0);
  }
  return r;
}

template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> operator-(const Tan<T, N, A>& x) {
  Tan<T, N, A> r;
  r.v = -x.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = has<A>(k) ? -x.d[k] : T(0);
  return r;
}

// Tan (op) passive scalar ---------------------------------------------------------
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> operator*(const Tan<T, N, A>& x, T c) {
  Tan<T, N, A> r;
  r.v = x.v * c;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = has<A>(k) ? x.d[k] * c : T(0);
  return r;
}
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> operator*(T c, const Tan<T, N, A>& x) { return x * c; }

template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> operator+(const Tan<T, N, A>& x, T c) {
  Tan<T, N, A> r = x;
  r.v = x.v + c;
  return r;
}
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> operator+(T c, const Tan<T, N, A>& x) { return x + c; }
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> operator-(const Tan<T, N, A>& x, T c) { return x + (-c); }
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> operator-(T c, const Tan<T, N, A>& x) { return (-x) + c; }

// Elementary functions on numbers: value and the chain rule for tangents.
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> chain(const Tan<T, N, A>& x, T f, T df) {
  Tan<T, N, A> r;
  r.v = f;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = has<A>(k) ? df * x.d[k] : T(0);
  return r;
}

AD_HD double inv(double x) { return 1.0 / x; }
AD_HD float inv(float x) { return 1.0f / x; }
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> inv(const Tan<T, N, A>& x) {
  const T r = inv(x.v);
  return chain(x, r, -r * r);
}

AD_HD double sqrt_(double x) { return std::sqrt(x); }
AD_HD float sqrt_(float x) { return sqrtf(x); }
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> sqrt_(const Tan<T, N, A>& x) {
  const T r = sqrt_(x.v);
  return chain(x, r, T(0.5) * inv(r));
}

AD_HD double exp_(double x) { return std::exp(x); }
AD_HD float exp_(float x) { return expf(x); }
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> exp_(const Tan<T, N, A>& x) {
  const T r = exp_(x.v);
  return chain(x, r, r);
}

AD_HD double log_(double x) { return std::log(x); }
AD_HD float log_(float x) { return logf(x); }
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> log_(const Tan<T, N, A>& x) { return chain(x, log_(x.v), inv(x.v)); }

// x^p for x > 0 and a passive exponent p.  FP64: the table-driven power of
// fpow.cuh (~26 FP64 operations; exp(p log x) takes ~54 FMA-equivalents and
// the general pow() ~98 on GB300, measured).  FP32: exp(p log x).
AD_HD double pow_(double x, double p) { return fpow::pow_pos(x, p); }
AD_HD float pow_(float x, float p) { return expf(p * logf(x)); }
template <class T, int N, unsigned A>
AD_HD Tan<T, N, A> pow_(const Tan<T, N, A>& x, T p) {
  const T r = pow_(x.v, p);
  if constexpr (sizeof(T) == 4) {
    // FP32: p x^(p-1) alone can overflow for tiny x where the product with
    // the tangent does not; scale the tangent by 1/x first
    const T ix = inv(x.v), pr = p * r;
    Tan<T, N, A> o;
    o.v = r;
#pragma unroll
    for (int k = 0; k < N; ++k) o.d[k] = has<A>(k) ? pr * (x.d[k] * ix) : T(0);
    return o;
  } else {
    // d/dx x^p at x = 0: 0 for p = 0 or p > 1, 1 for p = 1, unbounded for p < 1
    const T d = x.v != T(0) ? p * r * inv(x.v)
                            : (p == T(0) ? T(0) : p == T(1) ? T(1) : p > T(1) ? T(0) : T(INFINITY));
    return chain(x, r, d);
  }
}

// -------------------------------------------------------- adjoint accumulators

template <class V> struct adj_of { using type = V; };
template <class T, int N, unsigned M> struct adj_of<Tan<T, N, M>> {
  using type = Tan<T, N, (N >= 32 ? 0xffffffffu : ((1u << N) - 1u))>;
};

template <class T> AD_HD void set_neg_zero(T& a) { a = T(-0.0); }
template <class T, int N, unsigned M> AD_HD void set_neg_zero(Tan<T, N, M>& a) {
  a.v = T(-0.0);
#pragma unroll
  for (int k = 0; k < N; ++k) a.d[k] = T(-0.0);
}

AD_HD void accumulate(double& a, const double& b) { a = a + b; }
AD_HD void accumulate(float& a, const float& b) { a = a + b; }
template <class T, int N, unsigned F> AD_HD void accumulate(Tan<T, N, F>& a, const T& b) { a.v = a.v + b; }
template <class T, int N, unsigned F, unsigned B>
AD_HD void accumulate(Tan<T, N, F>& a, const Tan<T, N, B>& b) {
  a.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (has<B>(k)) a.d[k] = a.d[k] + b.d[k];
}

// ----------------------------------------------------------- expression nodes

template <class D> struct Expr {
  AD_HD const D& self() const { return *static_cast<const D*>(this); }
};

// Active leaf: holds the primal value and accumulates its adjoint.
template <class V> struct Var : Expr<Var<V>> {
  using value_type = V;
  using scalar = scalar_of_t<V>;
  using adj_type = typename adj_of<V>::type;
  V v;
  mutable adj_type a;
  AD_HD Var() { set_neg_zero(a); }
  AD_HD explicit Var(const V& x) : v(x) { set_neg_zero(a); }
  AD_HD const V& fwd() const { return v; }
  AD_HD const V& val() const { return v; }
  template <class B> AD_HD void back(const B& bv) const { accumulate(a, bv); }
};

// Passive leaf: a value that takes no adjoint.
template <class V> struct Cst : Expr<Cst<V>> {
  using value_type = V;
  using scalar = scalar_of_t<V>;
  V v;
  AD_HD Cst() {}
  AD_HD explicit Cst(const V& x) : v(x) {}
  AD_HD const V& fwd() const { return v; }
  AD_HD const V& val() const { return v; }
  template <class B> AD_HD void back(const B&) const {}
};

// Leaves are referenced, inner nodes copied (they are a handful of registers).
template <class E> struct hold { using type = E; };
template <class V> struct hold<Var<V>> { using type = const Var<V>&; };
template <class E> using hold_t = typename hold<E>::type;

template <class L, class R> struct Add : Expr<Add<L, R>> {
  using value_type = decltype(std::declval<typename L::value_type>() + std::declval<typename R::value_type>());
  using scalar = typename L::scalar;
  hold_t<L> l;
  hold_t<R> r;
  mutable value_type v;
  AD_HD Add(const L& a, const R& b) : l(a), r(b) {}
  AD_HD value_type fwd() const { v = l.fwd() + r.fwd(); return v; }
  AD_HD const value_type& val() const { return v; }
  template <class B> AD_HD void back(const B& bv) const { l.back(bv); r.back(bv); }
};

template <class L, class R> struct Sub : Expr<Sub<L, R>> {
  using value_type = decltype(std::declval<typename L::value_type>() - std::declval<typename R::value_type>());
  using scalar = typename L::scalar;
  hold_t<L> l;
  hold_t<R> r;
  mutable value_type v;
  AD_HD Sub(const L& a, const R& b) : l(a), r(b) {}
  AD_HD value_type fwd() const { v = l.fwd() - r.fwd(); return v; }
  AD_HD const value_type& val() const { return v; }
  template <class B> AD_HD void back(const B& bv) const { l.back(bv); r.back(-bv); }
};

template <class L, class R> struct Mul : Expr<Mul<L, R>> {
  using value_type = decltype(std::declval<typename L::value_type>() * std::declval<typename R::value_type>());
  using scalar = typename L::scalar;
  hold_t<L> l;
  hold_t<R> r;
  mutable value_type v;
  AD_HD Mul(const L& a, const R& b) : l(a), r(b) {}
  AD_HD value_type fwd() const { v = l.fwd() * r.fwd(); return v; }
  AD_HD const value_type& val() const { return v; }
  template <class B> AD_HD void back(const B& bv) const {
    l.back(bv * r.val());
    r.back(bv * l.val());
  }
};

// expression * passive scalar
template <class L> struct Scale : Expr<Scale<L>> {
  using value_type = typename L::value_type;
  using scalar = typename L::scalar;
  hold_t<L> l;
  scalar c;
  mutable value_type v;
  AD_HD Scale(const L& a, scalar s) : l(a), c(s) {}
  AD_HD value_type fwd() const { v = l.fwd() * c; return v; }
  AD_HD const value_type& val() const { return v; }
  template <class B> AD_HD void back(const B& bv) const { l.back(bv * c); }
};

// expression + passive scalar
template <class L> struct Shift : Expr<Shift<L>> {
  using value_type = typename L::value_type;
  using scalar = typename L::scalar;
  hold_t<L> l;
  scalar c;
  mutable value_type v;
  AD_HD Shift(const L& a, scalar s) : l(a), c(s) {}
  AD_HD value_type fwd() const { v = l.fwd() + c; return v; }
  AD_HD const value_type& val() const { return v; }
  template <class B> AD_HD void back(const B& bv) const { l.back(bv); }
};

template <class L> struct Neg : Expr<Neg<L>> {
  using value_type = typename L::value_type;
  using scalar = typename L::scalar;
  hold_t<L> l;
  mutable value_type v;
  AD_HD explicit Neg(const L& a) : l(a) {}
  AD_HD value_type fwd() const { v = -l.fwd(); return v; }
  AD_HD const value_type& val() const { return v; }
  template <class B> AD_HD void back(const B& bv) const { l.back(-bv); }
};

// Unary elementary operation.  F::f(x) gives the value, F::df(x, fx) the
// derivative expressed through the cached value fx; on Tan numbers df carries
// the second derivative along the tangent automatically.
template <class L, class F> struct Unary : Expr<Unary<L, F>> {
  using value_type = typename L::value_type;
  using scalar = typename L::scalar;
  hold_t<L> l;
  F op;
  mutable value_type v;
  AD_HD Unary(const L& a, F f) : l(a), op(f) {}
  AD_HD value_type fwd() const { v = op.f(l.fwd()); return v; }
  AD_HD const value_type& val() const { return v; }
  template <class B> AD_HD void back(const B& bv) const { l.back(bv * op.df(l.val(), v)); }
};

template <class T> struct FSqrt {
  template <class X> AD_HD X f(const X& x) const { return sqrt_(x); }
  template <class X> AD_HD X df(const X&, const X& r) const { return T(0.5) * inv(r); }
};
template <class T> struct FExp {
  template <class X> AD_HD X f(const X& x) const { return exp_(x); }
  template <class X> AD_HD X df(const X&, const X& r) const { return r; }
};
template <class T> struct FLog {
  template <class X> AD_HD X f(const X& x) const { return log_(x); }
  template <class X> AD_HD X df(const X& x, const X&) const { return inv(x); }
};
template <class T> struct FInv {
  template <class X> AD_HD X f(const X& x) const { return inv(x); }
  template <class X> AD_HD X df(const X&, const X& r) const { return -(r * r); }
};
template <class T> struct FSq {
  template <class X> AD_HD X f(const X& x) const { return x * x; }
  template <class X> AD_HD X df(const X& x, const X&) const { return x * T(2); }
};
// x^p for x > 0 and a passive exponent p.  The node caches w = x^(p-1):
// x^p = x w and d/dx = p w, so a first-order sweep needs no division (the
// second-order tangent of w carries the one reciprocal).
template <class L> struct PowN : Expr<PowN<L>> {
  using value_type = typename L::value_type;
  using scalar = typename L::scalar;
  hold_t<L> l;
  scalar p;
  mutable value_type v, w;
  AD_HD PowN(const L& a, scalar e) : l(a), p(e) {}
  AD_HD value_type fwd() const {
    const value_type x = l.fwd();
    w = pow_(x, p - scalar(1));
    v = x * w;
    return v;
  }
  AD_HD const value_type& val() const { return v; }
  template <class B> AD_HD void back(const B& bv) const { l.back(bv * (w * p)); }
};

// ------------------------------------------------------------------ operators

template <class A, class B> AD_HD Add<A, B> operator+(const Expr<A>& a, const Expr<B>& b) {
  return Add<A, B>(a.self(), b.self());
}
template <class A, class B> AD_HD Sub<A, B> operator-(const Expr<A>& a, const Expr<B>& b) {
  return Sub<A, B>(a.self(), b.self());
}
template <class A, class B> AD_HD Mul<A, B> operator*(const Expr<A>& a, const Expr<B>& b) {
  return Mul<A, B>(a.self(), b.self());
}
template <class A> AD_HD Scale<A> operator*(const Expr<A>& a, typename A::scalar c) { return Scale<A>(a.self(), c); }
template <class A> AD_HD Scale<A> operator*(typename A::scalar c, const Expr<A>& a) { return Scale<A>(a.self(), c); }
template <class A> AD_HD Scale<A> operator/(const Expr<A>& a, typename A::scalar c) {
  return Scale<A>(a.self(), typename A::scalar(1) / c);
}
template <class A> AD_HD Shift<A> operator+(const Expr<A>& a, typename A::scalar c) { return Shift<A>(a.self(), c); }
template <class A> AD_HD Shift<A> operator+(typename A::scalar c, const Expr<A>& a) { return Shift<A>(a.self(), c); }
template <class A> AD_HD Shift<A> operator-(const Expr<A>& a, typename A::scalar c) { return Shift<A>(a.self(), -c); }
template <class A> AD_HD Neg<A> operator-(const Expr<A>& a) { return Neg<A>(a.self()); }
template <class A> AD_HD Shift<Neg<A>> operator-(typename A::scalar c, const Expr<A>& a) {
  return Shift<Neg<A>>(Neg<A>(a.self()), c);
}
template <class A, class B>
AD_HD Mul<A, Unary<B, FInv<typename B::scalar>>> operator/(const Expr<A>& a, const Expr<B>& b) {
  return Mul<A, Unary<B, FInv<typename B::scalar>>>(a.self(), Unary<B, FInv<typename B::scalar>>(b.self(), {}));
}

template <class A> AD_HD Unary<A, FSqrt<typename A::scalar>> sqrt(const Expr<A>& a) { return {a.self(), {}}; }
template <class A> AD_HD Unary<A, FExp<typename A::scalar>> exp(const Expr<A>& a) { return {a.self(), {}}; }
template <class A> AD_HD Unary<A, FLog<typename A::scalar>> log(const Expr<A>& a) { return {a.self(), {}}; }
template <class A> AD_HD Unary<A, FSq<typename A::scalar>> sq(const Expr<A>& a) { return {a.self(), {}}; }
template <class A> AD_HD PowN<A> pow(const Expr<A>& a, typename A::scalar p) { return PowN<A>(a.self(), p); }

// sqrt whose derivative at 0 is taken as 0: for the norm of a generalized
// stress whose zero lies inside an elastic domain, where the adjoint that
// arrives is 0 and 0 * inf must not turn into NaN.
template <class T> struct FSqrt0 {
  // a forward tangent carried through x = 0 stays 0 (sqrt_ of a tangent type
  // would divide it by 2 sqrt(0))
  template <class X> AD_HD X f(const X& x) const { return value_of(x) > T(0) ? sqrt_(x) : x * T(0); }
  template <class X> AD_HD X df(const X&, const X& r) const {
    return value_of(r) > T(0) ? T(0.5) * inv(r) : r * T(0);
  }
};
// (x^+)^m, m >= 1: the power of the positive part (a yield function's overstress).
template <class T> struct FPosPow {
  T m;
  template <class X> AD_HD X f(const X& x) const { return value_of(x) > T(0) ? pow_(x, m) : x * T(0); }
  template <class X> AD_HD X df(const X& x, const X&) const {
    return value_of(x) > T(0) ? m * pow_(x, m - T(1)) : x * T(0);
  }
};
template <class A> AD_HD Unary<A, FSqrt0<typename A::scalar>> sqrt0(const Expr<A>& a) { return {a.self(), {}}; }
template <class A> AD_HD Unary<A, FPosPow<typename A::scalar>> pospow(const Expr<A>& a, typename A::scalar m) {
  return {a.self(), {m}};
}

// ------------------------------------------------- structural second order
// Which tangent components can reach a leaf's adjoint in a forward-over-reverse
// sweep, read off the expression's type: a node passes its incoming adjoint's
// mask down, a product adds the other factor's value mask, a nonlinear unary
// node its argument's.  For leaves seeded with unit tangents (mask 1 << k) the
// result is the structural pattern of the Hessian row of that leaf: the sweep
// leaves every other component at its initial -0.0.  Kernels use it to skip the
// structural zeros of constant Hessian blocks at compile time.
template <class V> constexpr unsigned vmask_of() {
  if constexpr (tan_info<V>::is_tan) return tan_info<V>::mask;
  else return 0u;
}
template <class E> constexpr unsigned vmask() { return vmask_of<typename E::value_type>(); }

template <unsigned LM, class E> struct Reach;
template <unsigned LM, class V> struct Reach<LM, Var<V>> {
  static constexpr unsigned at(unsigned in) { return vmask_of<V>() == LM ? in : 0u; }
};
template <unsigned LM, class V> struct Reach<LM, Cst<V>> {
  static constexpr unsigned at(unsigned) { return 0u; }
};
template <unsigned LM, class L, class R> struct Reach<LM, Add<L, R>> {
  static constexpr unsigned at(unsigned in) { return Reach<LM, L>::at(in) | Reach<LM, R>::at(in); }
};
template <unsigned LM, class L, class R> struct Reach<LM, Sub<L, R>> {
  static constexpr unsigned at(unsigned in) { return Reach<LM, L>::at(in) | Reach<LM, R>::at(in); }
};
template <unsigned LM, class L, class R> struct Reach<LM, Mul<L, R>> {
  static constexpr unsigned at(unsigned in) {
    return Reach<LM, L>::at(in | vmask<R>()) | Reach<LM, R>::at(in | vmask<L>());
  }
};
template <unsigned LM, class L> struct Reach<LM, Scale<L>> {
  static constexpr unsigned at(unsigned in) { return Reach<LM, L>::at(in); }
};
template <unsigned LM, class L> struct Reach<LM, Shift<L>> {
  static constexpr unsigned at(unsigned in) { return Reach<LM, L>::at(in); }
};
template <unsigned LM, class L> struct Reach<LM, Neg<L>> {
  static constexpr unsigned at(unsigned in) { return Reach<LM, L>::at(in); }
};
template <unsigned LM, class L, class F> struct Reach<LM, Unary<L, F>> {
  static constexpr unsigned at(unsigned in) { return Reach<LM, L>::at(in | vmask<L>()); }
};
template <unsigned LM, class L> struct Reach<LM, PowN<L>> {
  static constexpr unsigned at(unsigned in) { return Reach<LM, L>::at(in | vmask<L>()); }
};
// Polynomial degree of an expression in its active (tangent-carrying) leaves,
// read off its type; kNonPoly for anything a polynomial cannot express.  A
// degree <= 2 certifies that the Hessian does not depend on the point.
constexpr int kNonPoly = 1 << 20;
constexpr int deg_max(int a, int b) { return a > b ? a : b; }
constexpr int deg_mul(int a, int b) { return (a >= kNonPoly || b >= kNonPoly) ? kNonPoly : a + b; }
template <class E> struct Degree;
template <class V> struct Degree<Var<V>> { static constexpr int value = vmask_of<V>() ? 1 : 0; };
template <class V> struct Degree<Cst<V>> { static constexpr int value = vmask_of<V>() ? 1 : 0; };
template <class L, class R> struct Degree<Add<L, R>> {
  static constexpr int value = deg_max(Degree<L>::value, Degree<R>::value);
};
template <class L, class R> struct Degree<Sub<L, R>> {
  static constexpr int value = deg_max(Degree<L>::value, Degree<R>::value);
};
template <class L, class R> struct Degree<Mul<L, R>> {
  static constexpr int value = deg_mul(Degree<L>::value, Degree<R>::value);
};
template <class L> struct Degree<Scale<L>> { static constexpr int value = Degree<L>::value; };
template <class L> struct Degree<Shift<L>> { static constexpr int value = Degree<L>::value; };
template <class L> struct Degree<Neg<L>> { static constexpr int value = Degree<L>::value; };
template <class L, class T> struct Degree<Unary<L, FSq<T>>> {
  static constexpr int value = deg_mul(Degree<L>::value, Degree<L>::value);
};
template <class L, class F> struct Degree<Unary<L, F>> {
  static constexpr int value = Degree<L>::value == 0 ? 0 : kNonPoly;
};
template <class L> struct Degree<PowN<L>> { static constexpr int value = Degree<L>::value == 0 ? 0 : kNonPoly; };

// Hessian row pattern of the leaf seeded 1 << k in expression E (root adjoint 1).
template <class E, int K> constexpr unsigned hess_row() { return Reach<(1u << K), E>::at(0u); }

// ---------------------------------------------------------------- leaf packs
// A heterogeneous, fixed-size set of leaves addressed by a compile-time index:
// leaf k may carry its own tangent mask (unit seed e_k).

template <int I, class L> struct Slot { L leaf; };
template <class Seq, class... Ls> struct PackImpl;
template <int... Is, class... Ls>
struct PackImpl<std::integer_sequence<int, Is...>, Ls...> : Slot<Is, Ls>... {
  static constexpr int size = sizeof...(Ls);
};
template <class... Ls> using Pack = PackImpl<std::make_integer_sequence<int, sizeof...(Ls)>, Ls...>;

template <int I, class L> AD_HD const L& get(const Slot<I, L>& s) { return s.leaf; }
template <int I, class L> AD_HD L& get_mut(Slot<I, L>& s) { return s.leaf; }

// Compile-time loop helper.
template <int B, int E> struct For {
  template <class F> AD_HD static void run(F&& f) {
    if constexpr (B < E) {
      f(std::integral_constant<int, B>{});
      For<B + 1, E>::run(f);
    }
  }
};

// Pack of K leaves of kind LeafT<V_k>; V_k = Tan<T, N, 1 << (OFF + k)> (unit seeds).
template <template <class> class LeafT, class T, int N, int OFF, class Seq> struct SeededPackT;
template <template <class> class LeafT, class T, int N, int OFF, int... Is>
struct SeededPackT<LeafT, T, N, OFF, std::integer_sequence<int, Is...>> {
  using type = Pack<LeafT<Tan<T, N, (1u << (OFF + Is))>>...>;
};
template <template <class> class LeafT, class T, int N, int OFF, int K>
using SeededPack = typename SeededPackT<LeafT, T, N, OFF, std::make_integer_sequence<int, K>>::type;

template <class L, class Seq> struct UniformPackT;
template <class L, int... Is> struct UniformPackT<L, std::integer_sequence<int, Is...>> {
  template <int> using same = L;
  using type = Pack<same<Is>...>;
};
template <class L, int K> using UniformPack = typename UniformPackT<L, std::make_integer_sequence<int, K>>::type;

// Fill a seeded pack: value x[k], tangent component OFF+k set to 1.
template <class P, class T, int OFF, int K> AD_HD void seed_unit(P& p, const T* x) {
  For<0, K>::run([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    auto& leaf = get_mut<k>(p);
    leaf.v.v = x[k];
#pragma unroll
    for (int j = 0; j < sizeof(leaf.v.d) / sizeof(T); ++j) leaf.v.d[j] = T(0);
    leaf.v.d[OFF + k] = T(1);
  });
}

}  // namespace ad
}  // namespace gsm
