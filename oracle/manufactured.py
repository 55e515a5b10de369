"""Manufactured solution of the sphere accuracy benchmark (paper Sec. 4; oracle, test
infrastructure only).

On the ball of radius R around c, with r = |x - c| and d the dimension,
    u(r) = cos(omega R) - cos(omega r),
    f(r) = -omega^2 (cos(omega r) + (d - 1) sinc(omega r)),   sinc(z) = sin(z) / z, sinc(0) = 1,
satisfy -Lap u = f in the ball and u = 0 on the sphere (the Dirichlet data g = 0 that the Nitsche
terms impose).  The paper leaves omega open.
"""
import numpy as np


def _r(X, c):
    return np.sqrt(np.sum((np.asarray(X) - np.asarray(c)[None, :]) ** 2, axis=1))


def solution(X, c, R, omega):
    return np.cos(omega * R) - np.cos(omega * _r(X, c))


def rhs(X, c, R, omega):
    d = np.asarray(X).shape[1]
    z = omega * _r(X, c)
    sinc = np.where(z == 0.0, 1.0, np.sin(z) / np.where(z == 0.0, 1.0, z))
    return -omega ** 2 * (np.cos(z) + (d - 1) * sinc)
