"""GB300-native VEGAS iteration (sm_103a CUDA behind a C-ABI library).

The native library is loaded on first use by :mod:`._native`; importing this
package alone (for example to reach :mod:`.workloads`) loads no CUDA code.
"""
__all__ = ["workloads"]
