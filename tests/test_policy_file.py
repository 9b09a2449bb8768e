"""fbpt_policy_load rejects files that are not a policy before it touches the
device: a missing file, a token that is not a number, too few or too many
numbers.  No GPU."""
import numpy as np
import pytest

import paper_2311_10201_gb300 as fbpt


@pytest.fixture(scope="module", autouse=True)
def built():
    fbpt.build()


def load_code(path):
    with pytest.raises(fbpt.FbptError) as ei:
        fbpt.Policy.load(path)
    return ei.value.code


def test_bad_policy_files_rejected(tmp_path):
    count = fbpt.lib().fbpt_policy_param_count()
    assert load_code(tmp_path / "missing.txt") == fbpt.EINVAL
    short = tmp_path / "short.txt"
    np.savetxt(short, np.ones(count - 1, np.float32))
    assert load_code(short) == fbpt.EINVAL
    long = tmp_path / "long.txt"
    np.savetxt(long, np.ones(count + 1, np.float32))
    assert load_code(long) == fbpt.EINVAL
    word = tmp_path / "word.txt"
    word.write_text("1.0\n" * (count - 1) + "abc\n")
    assert load_code(word) == fbpt.EINVAL
