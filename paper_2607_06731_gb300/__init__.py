"""GB300-native population fitness scoring for Beagle-style postfix programs."""
