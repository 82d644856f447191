// zeus_user_objectives.cuh -- the default plug-in of user objectives
// (contract in include/zeus_user.cuh): two test functions that are not
// among the built-in ones, written once for every scalar type so that
// forward mode differentiates them (Alg. 5).  The build compiles another
// plug-in in its place when one is given.
#pragma once

#include "zeus_user.cuh"

#define ZEUS_USER_COUNT 2

namespace zeus_user {

// Griewank: 1 + (1/4000) sum_i x_i^2 - prod_i cos(x_i / sqrt(i)), i = 1..d.
// Global minimum 0 at the origin; the product couples every coordinate.
template <>
struct objective<0> {
    static constexpr const char* name = "griewank";
    static constexpr int min_dim = 1;
    static constexpr int max_dim = 0;

    template <class S, class X>
    __device__ static S eval(const X& x, int d) {
        using R = scalar_t<S>;
        S sum = S(0), prod = S(1);
        for (int j = 0; j < d; ++j) {
            const S xj = x(j);
            sum = sum + xj * xj;
            prod = prod * cos(xj / sqrt(R(j + 1)));
        }
        return (S(1) + sum / R(4000)) - prod;
    }
};

// Himmelblau: (x^2 + y - 11)^2 + (x + y^2 - 7)^2, d = 2.  Four global
// minima with value 0, one of them at (3, 2).
template <>
struct objective<1> {
    static constexpr const char* name = "himmelblau";
    static constexpr int min_dim = 2;
    static constexpr int max_dim = 2;

    template <class S, class X>
    __device__ static S eval(const X& x, int) {
        using R = scalar_t<S>;
        const S a = (x(0) * x(0) + x(1)) - R(11);
        const S b = (x(0) + x(1) * x(1)) - R(7);
        return a * a + b * b;
    }
};

}  // namespace zeus_user
