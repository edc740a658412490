import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_golden(name):
    import json
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        return json.load(f)


# Mutation tests (tests/test_oracle_mutants.py) rerun the oracle's pins in a
# child pytest against a deliberately broken copy of the oracle, named here.
_MUTANT_LIB = os.environ.get("ORACLE_MUTANT_LIB")
_MUTANT_MLP = os.environ.get("ORACLE_MUTANT_MLP")
if _MUTANT_LIB or _MUTANT_MLP:
    import oracle

    if _MUTANT_LIB:
        oracle._lib = oracle.load(_MUTANT_LIB)
    if _MUTANT_MLP:
        import importlib.util

        spec = importlib.util.spec_from_file_location("oracle.mlp", _MUTANT_MLP)
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        sys.modules["oracle.mlp"] = mod
        oracle.mlp = mod
