"""Helpers shared by the GPU tests: tolerances and argument builders.

Tolerances (floating point, against the FP64 oracle):
  bn mean   |d| <= 1e-5 * mean_c(|x|)          (summation conditioning scale)
  bn var    |d| <= 1e-4 * var_c                 (relative)
  upsample  |d| <= 1e-5 * |ref|                 (relative; inputs >= 0)
  poly      |d| <= 1e-5 * (|ref| + bound)       (Horner conditioning scale)
  stream    |d| <= 1e-5 * max(|ref|, |x|, 1)
  bf16      at most 1 bf16 ulp
Integer, copy and max work is compared bit for bit.
"""
import numpy as np
import torch

import oracle
from paper_2007_01277_gb300 import hfuse as H
from paper_2007_01277_gb300 import workloads as W

DEV = torch.device("cuda:0")


def check_bn(x_cpu, mean, var):
    m_ref, v_ref = oracle.bn_stats(x_cpu.numpy())
    xs = x_cpu.double().abs().transpose(0, 1).reshape(x_cpu.shape[1], -1).mean(1).numpy()
    m = mean.double().cpu().numpy()
    v = var.double().cpu().numpy()
    assert np.all(np.abs(m - m_ref) <= 1e-5 * xs + 1e-30), np.max(np.abs(m - m_ref) / xs)
    assert np.all(np.abs(v - v_ref) <= 1e-4 * v_ref + 1e-12), np.max(np.abs(v - v_ref) / v_ref)


def check_upsample(x_cpu, y):
    ref = oracle.upsample2x(x_cpu.numpy())
    got = y.double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-30), np.max(np.abs(got - ref))


def check_poly(x_cpu, coef, y, iters=64):
    ref, bound = oracle.poly(x_cpu.numpy(), coef, iters=iters, with_bound=True)
    got = y.double().cpu().numpy()
    err = np.abs(got - ref) / (np.abs(ref) + bound + 1e-300)
    assert np.all(err <= 1e-5), err.max()


def check_stream(x_cpu, y, k, a, b):
    ref = oracle.stream_tmpl(x_cpu.numpy(), k, a, b)
    got = y.double().cpu().numpy()
    scale = np.maximum(np.maximum(np.abs(ref), np.abs(x_cpu.double().numpy())), 1.0)
    assert np.all(np.abs(got - ref) <= 1e-5 * scale), np.max(np.abs(got - ref) / scale)


def bits16(t):
    return t.view(torch.int16).cpu().numpy().view(np.uint16)


def check_bf16(x_cpu, y_cpu, out, alpha=0.5):
    ref = oracle.bf16_axpy(bits16(x_cpu), bits16(y_cpu), alpha)
    got = bits16(out)
    # bf16 bit patterns of same-sign finite values are ordered: 1 ulp = 1 step
    diff = np.abs(got.astype(np.int32) - ref.astype(np.int32))
    assert np.all(diff <= 1), diff.max()
    return int((diff != 0).sum())


def single(body, args, threads, grid):
    k = H.hf_register_kernel(body)
    H.hf_launch_single(k, args, threads, grid)
    return k
