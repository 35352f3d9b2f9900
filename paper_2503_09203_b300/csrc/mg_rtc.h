// Base types and the few type traits the kernel headers use, for both of
// their compilers: nvcc (the library's own build) and NVRTC (the run-time
// compiler that builds class-specialised step kernels; it compiles these
// headers without the host C/C++ library).
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
namespace mg {
namespace tt {
template <class A, class B> struct is_same { static constexpr bool value = false; };
template <class A> struct is_same<A, A> { static constexpr bool value = true; };
template <bool C, class T, class F> struct conditional { using type = T; };
template <class T, class F> struct conditional<false, T, F> { using type = F; };
template <bool C, class T, class F> using conditional_t = typename conditional<C, T, F>::type;
template <class T> struct remove_ref { using type = T; };
template <class T> struct remove_ref<T&> { using type = T; };
template <class T> struct remove_ref<T&&> { using type = T; };
template <class T> struct remove_cv { using type = T; };
template <class T> struct remove_cv<const T> { using type = T; };
template <class T> struct remove_cv<volatile T> { using type = T; };
template <class T> struct remove_cv<const volatile T> { using type = T; };
template <class T> using decay_t = typename remove_cv<typename remove_ref<T>::type>::type;
}  // namespace tt
}  // namespace mg
#else
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>
namespace mg {
namespace tt {
using std::conditional_t;
using std::decay_t;
using std::is_same;
}  // namespace tt
}  // namespace mg
#endif
